/*
 * libpfire — GB300 (sm_103a) library for the wildfire cellular automaton of
 * arXiv 2502.18738 (PyTorchFire): the per-step 8-neighbour stencil in its discrete
 * stochastic form and its differentiable (mean-field) form, and the reverse-time
 * adjoint of the differentiable form.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Grid H x W, row-major, row r grows southward, column c grows eastward. Every
 *   per-cell array passed in or out is dense: element (r, c) at offset r*W + c, and a
 *   batch of R realisations is R consecutive H*W planes.
 * - Unless stated otherwise, array pointers are DEVICE pointers owned by the caller
 *   and valid for the duration of the call (inputs are copied into library-owned
 *   buffers before the call returns to the stream, so the caller may reuse them once
 *   the stream has passed the call). Outputs are caller-allocated device memory.
 * - All work is enqueued on the CUDA stream given to pf_create; calls return before
 *   the work finishes unless stated otherwise ("synchronous").
 * - Discrete states are uint8: 0 non-burnable, 1 unburned (burnable), 2 burning,
 *   3 burned (Sec. 2.2, "State and transition rules"; the paper's non-burnable
 *   "no forest fuel" state is kept as its own code).
 * - Directions: the burning neighbour i of a receiving cell j sits at offset
 *   (dr, dc) in the fixed order (-1,-1) (-1,0) (-1,1) (0,-1) (0,1) (1,-1) (1,0) (1,1).
 * - Every entry point returns a pf_status; on failure pf_last_error(ctx) holds a
 *   one-line message. A failed call leaves the context usable unless it returns
 *   PF_ECUDA, after which the CUDA context itself may be unusable.
 */
#ifndef PFIRE_H
#define PFIRE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pf_ctx pf_ctx;

typedef enum pf_status {
    PF_OK = 0,
    PF_EINVAL = -1,   /* bad argument: sizes, NULL where required, out-of-range values */
    PF_ENOMEM = -2,   /* device allocation failed */
    PF_ECUDA = -3,    /* a CUDA call or kernel launch failed */
    PF_ESTATE = -4,   /* call not valid in the context's current state */
    PF_ETIMEOUT = -5  /* a bounded device wait ran out (batched kernel) */
} pf_status;

typedef enum pf_form {
    PF_DISCRETE = 0,  /* stochastic uint8 automaton with Philox draws */
    PF_DIFF = 1       /* differentiable continuous-state form, FP32 (a, b) */
} pf_form;

/* Create a context for an H x W grid.
 *   form          PF_DISCRETE or PF_DIFF.
 *   realisations  R >= 1 independent stochastic runs sharing one landscape (discrete
 *                 form); must be 1 for PF_DIFF, which is deterministic.
 *   seed          64-bit Philox key (Sec. 2.2 data flow: "two random matrices").
 *   cuda_stream   cudaStream_t to run on (NULL = legacy default stream).
 * Limits: 1 <= H, W <= 65536, H*W*R < 2^32. Allocates the state and q buffers; the
 * landscape defaults to flat, calm, p_veg = p_den = 0, parameters to the paper's
 * calibration start values (p_h 0.58, c1 0.045, c2 0.131, a 0.078, p_continue 0.3,
 * l 30 m). Returns PF_EINVAL / PF_ENOMEM / PF_ECUDA; *out is NULL on failure. */
int pf_create(pf_ctx** out, int H, int W, int form, int realisations, uint64_t seed, void* cuda_stream);

/* Release every buffer of the context (synchronises its stream first). NULL is a no-op. */
void pf_destroy(pf_ctx* ctx);

/* Static landscape (Sec. 2.1 inputs): elevation E (m; the slope of Eq. 1 is derived
 * from it), vegetation p_veg and density p_den (Eq. 2), and the first wind epoch
 * (V_w m/s, theta_w degrees counter-clockwise from East, Eq. 3), which applies from
 * step 0. Each is an H*W FP32 device array; NULL selects the neutral factor, as the
 * paper's "empty tensor" rule does (flat terrain, p_veg = p_den = 0, no wind).
 * Returns PF_EINVAL if any p_veg or p_den is below -1 or any value is NaN or infinite.
 * Replaces all wind epochs. Synchronous validation (one device reduction). */
int pf_set_env(pf_ctx* ctx, const float* E, const float* p_veg, const float* p_den,
               const float* V_w, const float* theta_w_deg);

/* Slope given directly (Sec. 2.1: an H x W x 3 x 3 tensor of the slope from each cell to
 * its neighbours, degrees): slope_deg device FP32 [H][W][3][3], entry [r][c][dr+1][dc+1]
 * is Eq. 1's theta_s with E the cell (r, c) and E-hat its neighbour (r+dr, c+dc), i.e.
 * the slope of spread into (r, c) from that neighbour (the centre entry is unused). It
 * replaces the slopes derived from E until cleared with NULL. Copied. PF_EINVAL for
 * NaN / inf. */
int pf_set_slope(pf_ctx* ctx, const float* slope_deg);

/* Add a wind epoch (Eq. 3 inputs) that applies from global step from_step onwards,
 * until the next epoch. from_step must be > 0 and larger than every earlier epoch's;
 * NULL V_w means calm. V_w / theta_w_deg are H*W FP32 device arrays, copied into the
 * context (8 bytes per cell per epoch) after a synchronous validation (PF_EINVAL for
 * NaN / inf). Used to resample the wind during a run and replayed by pf_backward. */
int pf_set_wind(pf_ctx* ctx, const float* V_w, const float* theta_w_deg, int from_step);

/* pf_set_wind without blocking the host, for streaming the wind of later epochs while
 * a run computes. V_w / theta_w_deg are H*W FP32 arrays in host memory (page-locked,
 * for the copy to overlap; pageable memory works but is staged synchronously) or in
 * device memory. The copy runs on a stream of the context's own, after the work already
 * queued on the context's stream (the epoch's buffer may be one it released), and the
 * context's stream waits for it only when a kernel first reads the epoch. The caller
 * keeps the arrays valid and unchanged until the next pf_wait, pf_backward or
 * pf_destroy returns. The values are checked on the device: NaN or infinite values are
 * reported as PF_EINVAL by that next synchronising call, and the results of the runs
 * that read the epoch are then undefined. Returns PF_EINVAL at once for an out-of-order
 * from_step, PF_ENOMEM / PF_ECUDA. */
int pf_set_wind_async(pf_ctx* ctx, const float* V_w, const float* theta_w_deg, int from_step);

/* Wait for everything queued on the context (its stream and its upload stream) and
 * report what the device recorded since the last report: PF_ETIMEOUT if a bounded
 * device-side wait ran out, else PF_EINVAL for invalid values in an epoch uploaded by
 * pf_set_wind_async. Each condition is cleared once reported. */
int pf_wait(pf_ctx* ctx);

/* Model parameters (Sec. 2.1 list; Eq. 2-4): p_h base probability, c1 wind-speed
 * factor, c2 wind-direction factor, a slope factor (per degree), p_continue
 * probability that a burning cell keeps burning, l cell side in metres (Eq. 1).
 * Requires finite values, p_h >= 0, 0 <= p_continue <= 1 and l > 0 (else PF_EINVAL). */
int pf_set_params(pf_ctx* ctx, float p_h, float c1, float c2, float a, float p_continue, float l_m);

/* Run T >= 0 steps from S_init (uint8 [R][H][W], device), starting at global step 0.
 *   Discrete form: S_out is uint8 [R][H][W]. Realisation r draws with run index r.
 *   Differentiable form: S_init's codes map to a = [S in {2,3}], b = [S == 2]; code 0
 *   cells are non-burnable for the whole run. S_out is FP32 [2][H][W]: a_T (probability
 *   of having ignited by step T, the burn probability) then b_T (probability of burning).
 *   The run is recorded for pf_backward: (a, b) checkpoints every K steps (K chosen to
 *   fit free HBM, see pf_tuning) and the wind epochs it used.
 * S_out may be NULL (the state is kept in the context; see pf_get_state).
 * Sec. 2.2 transition rules and Eq. 9 for the discrete form; Eq. 9 with burning
 * probabilities in place of the burning indicator for the differentiable form. */
int pf_forward(pf_ctx* ctx, const uint8_t* S_init, int T, void* S_out);

/* Continue the current state for T more steps (same output layout as pf_forward).
 * Global step numbering continues, so pf_forward(T1) then pf_advance(T2) draws the
 * same numbers as pf_forward(T1 + T2). In the differentiable form the recorded run
 * is extended as well. */
int pf_advance(pf_ctx* ctx, int T, void* S_out);

/* Reverse-time adjoint of the last recorded differentiable run (PF_DIFF only; else,
 * or before any pf_forward, PF_ESTATE).
 *   dL_da_T, dL_db_T  FP32 [H][W] device gradients of the loss w.r.t. a_T and b_T
 *                     (either may be NULL = zero).
 *   grad_params       HOST double[4], overwritten with dL/d(p_h, c1, c2, a): the
 *                     parameter gradients summed over all cells and steps in FP64,
 *                     in a fixed order (bit-reproducible run to run).
 *   grad_pveg, grad_pden  FP32 [H][W] device outputs (nullable): dL/dp_veg, dL/dp_den
 *                     per cell (0 at non-burnable cells).
 * Recomputes each checkpoint segment, newest first, then sweeps it backwards.
 * Synchronous (grad_params is on the host when it returns); reports what pf_wait
 * reports. */
int pf_backward(pf_ctx* ctx, const float* dL_da_T, const float* dL_db_T, double grad_params[4],
                float* grad_pveg, float* grad_pden);

/* Current state and its global step number. S: discrete uint8 [R][H][W]; differentiable
 * FP32 [2][H][W] (a then b; the library keeps a and b down to about 1e-327, and values
 * below FP32's range are returned as their FP32 rounding, down to 0). step may be NULL. */
int pf_get_state(pf_ctx* ctx, int* step, void* S);

/* Overwrite the current state and set the global step counter (resume, and the
 * paper's in-place edits for spotting, Sec. 2.2). Discrete: uint8 [R][H][W] with codes
 * 0-3. Differentiable: FP32 [2][H][W] with 0 <= b <= a <= 1 (not validated); cells with
 * a == b == 0 remain burnable. Discards the recorded run. */
int pf_set_state(pf_ctx* ctx, int step, const void* S);

/* Counts of the current state, and the near-ties of the discrete draws (Sec. 2.2: the
 * transition compares p_ignite and p_continue with two random matrices; a cell whose
 * draw lies within 1e-6 of the probability it is compared with is a near-tie, the only
 * kind of cell whose transition may legitimately differ from the FP64 oracle's).
 *   step                 the current global step.
 *   cells[4]             discrete: cells in state 0, 1, 2, 3 over all realisations.
 *                        Differentiable: non-burnable cells, the expected unburned
 *                        cells (sum of 1 - a over burnable cells), the expected burning
 *                        cells (sum of b) and the expected burned cells (sum of a - b),
 *                        summed in FP64 in no fixed order.
 *   near_ties_ignite     discrete: unburned cells with a burning neighbour whose
 *                        ignition draw u satisfied |u - p_ignite| < 1e-6 (FP32 values),
 *                        over every step and realisation since the last pf_forward
 *                        (pf_advance adds to it). 0 in the differentiable form.
 *   near_ties_continue   the same for burning cells and |u - p_continue| < 1e-6.
 * Synchronous (reads the counts back); out is a host struct. */
typedef struct pf_stats_t {
    int step;
    double cells[4];
    long long near_ties_ignite;
    long long near_ties_continue;
} pf_stats_t;
int pf_stats(pf_ctx* ctx, pf_stats_t* out);

/* Ignition probability map p_ignite (Eq. 9) of the current state: FP32 [R][H][W]
 * (discrete: over burning neighbours, for every cell; differentiable: with burning
 * probabilities b, R = 1). The paper's real-time ignition-map accessor (Sec. 2.1). */
int pf_ignition_map(pf_ctx* ctx, float* P_out);

/* Binary cross-entropy of a burn-probability map against a 0/1 target, and its
 * gradient: yhat = clamp(a, 1e-7, 1 - 1e-7), L = -mean(y log yhat + (1-y) log(1-yhat)),
 * dL_da = (yhat - y) / (yhat (1 - yhat)) / n inside the clamp range, else 0.
 * a, y: FP32 [n] device; dL_da: FP32 [n] device (nullable); loss: HOST double
 * (nullable; if given the call is synchronous). Context-free; runs on cuda_stream. */
int pf_loss_bce(const float* a, const float* y, int64_t n, float* dL_da, double* loss, void* cuda_stream);

/* pf_loss_bce without any device allocation, for callers that may not allocate
 * device memory themselves or through the library: code whose device memory is owned
 * by an allocator with a fixed budget (a caching allocator or a reserved pool, where a
 * stray cudaMalloc fragments the pool or exceeds the budget), and latency-critical loops
 * in which the device-wide synchronisation of cudaMalloc / cudaFree is not acceptable.
 * The arithmetic and arguments are those of pf_loss_bce; the reduction scratch is a
 * statically allocated device array of 16385 doubles (128 KB, held by every GPU that
 * loads the library until the process exits), which bounds n to
 * PF_NOALLOC_BCE_MAX_N elements (larger n: PF_EINVAL, message via pf_last_error(NULL)).
 * The first call on a device looks up the array's device address (once per device and
 * context, with that device current); make that first call before any stream capture.
 * After cudaDeviceReset the next call looks the address up again in the new context. All calls share
 * the array: calls whose work overlaps on the GPU (different streams, or concurrent host
 * threads) race on it and must be serialised by the caller. Each call overwrites every
 * entry it reads, so no clearing is needed. The paper has no counterpart: this is a
 * deployment variant of pf_loss_bce. The loss may differ from pf_loss_bce's in the last
 * bits (a different block partition of the same FP64 reduction); dL_da is identical. */
#define PF_NOALLOC_BCE_MAX_N 67108864LL
int pf_loss_bce_noalloc(const float* a, const float* y, int64_t n, float* dL_da, double* loss, void* cuda_stream);

/* Kernel selection and checkpoint interval. Zero fields mean "choose automatically".
 *   kernel    1 = plain one-launch-per-step kernels, 2 = temporal-blocked TMA kernels.
 *   k         steps per launch of the temporal-blocked kernels (1..16; the differentiable
 *             kernels take at most 8, the discrete one at most 12).
 *   K         checkpoint interval of the differentiable form (>= 1; 1 keeps every state).
 *   profile   1 = time every kernel launch with CUDA events on the context's stream
 *             (read with pf_profile_read).
 *   prep      where the forward's ignition factors q (Eq. 1-5) come from: 1 = materialised
 *             once per wind epoch into eight FP32 planes that the step kernels read, 2 =
 *             recomputed inside the step kernels from the fields (the same arithmetic:
 *             results are identical). The adjoint always materialises q. 0 = 1.
 *   tile_rows interior rows per tile of the discrete blocked kernel (16, 32, 64 or 128; 0
 *             = 64); its halo is k rows (16 when k = 0). Ignored by the differentiable
 *             form, whose 64 x 64 regions take a 4-cell halo for k <= 4, else 8.
 *   tape      differentiable form with checkpoints (K > 1) and the blocked kernels:
 *             0 = keep a tile tape (every live tile's states of every forward launch)
 *             so that the backward copies each segment's states instead of recomputing
 *             them; a segment the tape does not cover is recomputed. The first tape
 *             takes the device memory the backward does not need, less a sixteenth of
 *             the device (at least 16 GB) left free, up to what T steps of every tile
 *             would take (18 KB a tile and step at the 8-cell halo); once a backward has
 *             seen how much the tape needs, it holds that and an eighth more. It is
 *             kept by the context until pf_destroy. The per-epoch q cache (the forward's q of every wind epoch
 *             kept for the adjoint) is kept beside it only where both fit; otherwise
 *             the backward prepares q again. 1 = no tape: always recompute.
 * Results do not depend on any of these (the same arithmetic in every variant), except
 * through K's effect on memory. PF_EINVAL for values out of range. */
typedef struct pf_tuning {
    int kernel;
    int k;
    int K;
    int profile;
    int prep;
    int tile_rows;
    int tape;
} pf_tuning;

int pf_set_tuning(pf_ctx* ctx, const pf_tuning* t);
int pf_get_tuning(const pf_ctx* ctx, pf_tuning* t);

/* Device memory the differentiable form's gradient path holds, and how the last taped
 * forward used it (no counterpart in the paper: memory planning for the checkpointed
 * backward). Bytes: checkpoint states (the arena), the backward's segment buffer, the
 * per-epoch q cache, the tile tape and the part of it the last taped forward wrote.
 * tape_launches: blocked launches of that forward the tape tried to record;
 * tape_recorded: those it had room for (the others are recomputed by the backward).
 * K: that forward's checkpoint interval; tape_short: the tape of the last backward
 * ran short (some of its launches were recomputed). allocations / frees: the device
 * allocations and frees the context has made so far (steady runs make none).
 * Synchronises the context's stream. */
typedef struct pf_memory_stats_t {
    long long checkpoint_bytes;
    long long segment_bytes;
    long long qcache_bytes;
    long long tape_bytes;
    long long tape_used_bytes;
    int tape_launches;
    int tape_recorded;
    int K;
    int tape_short;
    long long allocations;
    long long frees;
} pf_memory_stats_t;
int pf_memory_stats(pf_ctx* ctx, pf_memory_stats_t* out);

/* Autotuner (no counterpart in the paper, which has one PyTorch code path). Times, on
 * this context's grid, fields and parameters, a forward of T_probe steps from S_init
 * (device, uint8 [R][H][W] as for pf_forward) with each candidate launch configuration:
 * q materialised or recomputed (prep 1 / 2), each with the plain per-step kernels and
 * the temporal-blocked kernels at several depths k (differentiable: k in {2, 4, 6, 8};
 * discrete: k in {4, 8, 12} x tile_rows in {32, 64, 128}). Keeps the fastest as the
 * context's tuning (K and profile are left as they were) and writes the resulting
 * tuning to *chosen (nullable, host). The probe runs leave no tape: call pf_forward
 * before pf_backward.
 * On-disk cache: the choice is appended to a text file, one line per key (GPU model,
 * compute capability and SM count; form, H, W, R, T_probe), and a later call with the
 * same key applies the cached choice without timing. The file is $PF_TUNE_CACHE, else
 * $XDG_CACHE_HOME/pfire/tuning.tsv, else $HOME/.cache/pfire/tuning.tsv; PF_TUNE_CACHE
 * set to "" or "off" disables it. A file that cannot be read or written is skipped.
 * Synchronous. PF_EINVAL for NULL arguments, T_probe < 1 or invalid state codes. */
int pf_autotune(pf_ctx* ctx, const uint8_t* S_init, int T_probe, pf_tuning* chosen);

/* Checkpoint-interval search of the differentiable form (PF_DIFF only, else PF_ESTATE).
 * Times pf_forward of T steps from S_init plus pf_backward (zero loss gradients) for
 * the memory rule of pf_tuning.K = 0 and for intervals that are multiples of the
 * blocked kernels' k around the one it picks (launches are then never cut short at a
 * checkpoint), with the context's other tuning; keeps the fastest as pf_tuning.K (0 =
 * the memory rule) and writes it to *K_chosen (nullable, host). Uses the same on-disk
 * cache as pf_autotune (key: form, H, W, R, T). The probe runs leave no tape.
 * Synchronous; a candidate that does not fit in memory ends the search with PF_ENOMEM
 * and the tuning unchanged. */
int pf_autotune_ckpt(pf_ctx* ctx, const uint8_t* S_init, int T, int* K_chosen);

/* Per-kernel-kind launch counts, cell-steps processed (cells x automaton steps the
 * launches advanced or reversed), the part of those cell-steps the temporal-blocked
 * kernels skipped because their tile was quiescent (forward: b = 0 in the whole tile
 * region, so nothing changes; adjoint: a = 0 in the whole region, so lambda is 0; the
 * results are exact either way; for the kind "adjoint_tiles" it counts the cell-steps the
 * blocked adjoint ran on frozen tiles, whose region is constant over the launch; for
 * "diff_tiles" and "segment_tiles", the pre-passes of the blocked forward and of the
 * adjoint's segment recomputes, the cells they copied or zero-filled). The blocked
 * adjoint's frozen tiles run in a kernel of their own ("adjoint_frozen": its launches and
 * time; its cell-steps are those "adjoint_tiles" counts; "adjoint_blocked" counts every
 * cell-step of a launch, skipped = the void tiles') and, if
 * profiling, summed device milliseconds since the last reset. kinds[i] is a static name string; any output array may be NULL.
 * Synchronous. Returns the number of kinds written (<= max_kinds) or a negative pf_status. */
int pf_profile_read(pf_ctx* ctx, int max_kinds, const char** kinds, long long* launches, long long* cell_steps,
                    long long* skipped_cell_steps, double* ms, int reset);

/* ------------------------------------------- the paper's accumulator calibration path */

/* Accumulator of the discrete form (Sec. 2.2, data flow of Fig. 4: "the p_ignite values
 * of newly ignited cells are accumulated"). acc: device FP32 [R][H][W], caller-owned,
 * NULL disables. While set, pf_forward zero-fills it and records the trajectory (its
 * initial state, parameters and fields), and every step of pf_forward / pf_advance
 * writes into acc[r][j] the FP32 p_ignite (Eq. 9) with which cell j ignited; a cell
 * ignites at most once, and cells that never ignite (or burned from the start) keep 0.
 * PF_EINVAL for the differentiable form. */
int pf_set_accumulator(pf_ctx* ctx, float* acc);

/* Replace the Philox key of the context (the paper's model.reset() draws a new seed
 * per calibration epoch, Alg. 1). Invalidates recorded trajectories and tapes. */
int pf_reseed(pf_ctx* ctx, uint64_t seed);

/* Gradient of a loss of the accumulator (Sec. 2.3, back-propagation): with the sampled
 * trajectory held fixed, only the p_ignite of newly ignited cells depends on the
 * parameters, dp_ignite_j / dq_dj = beta_i prod_{e != d} (1 - beta_e q_ej) (beta: the
 * burning indicators of the step, Eq. 9), chained through Eq. 1-5 to (p_h, c1, c2, a)
 * and per-cell p_veg, p_den. The trajectory of the last pf_forward (+ pf_advance) with an
 * accumulator set is replayed from its initial state with the same Philox draws.
 *   dL_dacc     device FP32 [R][H][W]; realisations are summed.
 *   step_mask   host uint8 [steps run] or NULL (all): steps whose ignitions carry
 *               gradient (the paper's "step rings"); the others count as constants.
 *   grad_params host double[4]: dL/d(p_h, c1, c2, a), FP64 fixed-order reduction.
 *   grad_pveg, grad_pden  device FP32 [H][W] or NULL.
 * Synchronous. PF_ESTATE if no trajectory was recorded, or parameters, fields or wind
 * changed since it was. */
int pf_backward_dca(pf_ctx* ctx, const float* dL_dacc, const uint8_t* step_mask, double grad_params[4],
                    float* grad_pveg, float* grad_pden);

/* Loss of Eq. 10 on one H x W map: binary cross-entropy with logits of yhat against the
 * 0/1 observation y, averaged over the crop to the bounding box of the union of the
 * non-zero entries of yhat and y (the paper's acceleration; 0 if both are all zero),
 * plus the mean of (AvgPool(y) - AvgPool(yhat))^2 over the 4 x 4, stride-4 windows that
 * fit in the map. yhat, y: device FP32 [H][W]; dL_dyhat: device FP32 [H][W] or NULL;
 * loss: host double or NULL (then the call is asynchronous on cuda_stream). Block
 * partials are reduced in FP64 in a fixed order. */
int pf_loss_eq10(const float* yhat, const float* y, int H, int W, float* dL_dyhat, double* loss, void* cuda_stream);

/* ----------------------------------------------------------- ensemble metrics */

/* A cell is affected when its state is 2 (burning) or 3 (burned). All maps are device
 * uint8 state arrays; results are exact integer counts. */

/* Probability of arrival from an ensemble (the paper: "computed using an ensemble of
 * numerous CA runs ... by averaging these runs"): P_out[j] (device FP32 [H][W]) = the
 * fraction of the R realisations of S ([R][H][W]) in which cell j is affected. Async. */
int pf_arrival_probability(const uint8_t* S, int R, int H, int W, float* P_out, void* cuda_stream);

/* Affected cells of each of R maps of HW cells (S [R][HW]) into counts (host, R long
 * longs): the |A_t| of Eq. 12 for the state at one step. Synchronous. */
int pf_affected_count(const uint8_t* S, int R, int64_t HW, long long* counts, void* cuda_stream);

/* Manhattan distance of Eq. 12 between two runs: SA and SB are series of T maps of HW
 * cells ([T][HW] uint8, the state after each step); the affected counts |A_t| and
 * |Ahat_t| of every step are taken on the device and *out (host) receives the sum over t
 * of | |A_t| - |Ahat_t| |. Synchronous. */
int pf_manhattan(const uint8_t* SA, const uint8_t* SB, int T, int64_t HW, long long* out, void* cuda_stream);

/* Jaccard index of Eq. 11 between the affected sets of two maps of n cells:
 * |A and B| / |A or B|, 1 when both are empty. *out: host double. Synchronous. */
int pf_jaccard(const uint8_t* A, const uint8_t* B, int64_t n, double* out, void* cuda_stream);

/* ----------------------------------------------------------- batched fires */

/* One independent fire for pf_batch_submit. All pointers are device pointers; the
 * per-cell arrays are dense H*W FP32 (NULL = neutral factor, as in pf_set_env).
 *   form        PF_DISCRETE (S_out uint8 [H][W]) or PF_DIFF (S_out FP32 [2][H][W];
 *               the adjoint is not part of the batch).
 *   fire_id     Philox counter word 3, so fires draw disjoint streams.
 *   run         Philox counter word 1 (realisation index). */
typedef struct pf_job {
    int H, W, T, form;
    uint64_t seed;
    uint32_t run, fire_id;
    const float *E, *p_veg, *p_den, *V_w, *theta_w;
    float p_h, c1, c2, a, p_continue, l;
    const uint8_t* S_init;
    void* S_out;
    /* differentiable jobs only (all NULL: forward only). dL_da: device FP32 [H][W], the
     * gradient of a loss with respect to a_T; then grad_params (device double[4],
     * required) receives dL/d(p_h, c1, c2, a) and grad_pveg / grad_pden (device FP32
     * [H][W], nullable) the per-cell gradients, as pf_backward computes them. Every state
     * of such a job is kept on the device during the submission ((T + 1) x 8 B per cell). */
    const float* dL_da;
    double* grad_params;
    float *grad_pveg, *grad_pden;
} pf_job;

/* Run n independent fires of uneven sizes and step counts (each as pf_forward would,
 * bit-identically for the discrete form and the differentiable forward), with, for the
 * differentiable jobs that carry dL_da, their reverse-time adjoint and the parameter and
 * per-cell gradients. Jobs of at least pf_batch_set_direct_cells cells (default 2^18)
 * run one after another through a context of their own (the temporal-blocked kernels
 * and the context's automatic tuning, with the job's fire_id and run); the others from
 * one device work queue in a persistent kernel, then their adjoints from a second work
 * queue (block by block from each job's last step), in one captured CUDA graph per wave
 * of jobs that fits in memory. Synchronous. PF_ETIMEOUT if a bounded device-side wait
 * ran out, PF_ENOMEM if the states of the differentiable jobs with an adjoint do not fit. */
int pf_batch_submit(const pf_job* jobs, int n, void* cuda_stream);

/* Jobs of pf_batch_submit with H * W >= min_cells run through contexts of their own
 * (0: all of them; a value above every job's size: none). Process-wide; PF_EINVAL for
 * min_cells < 0. No counterpart in the paper (a scheduling choice of the batch). */
int pf_batch_set_direct_cells(long long min_cells);

/* Work and device time of this thread's last pf_batch_submit, summed over the waves it
 * ran in (jobs are grouped into waves that fit in free memory). Cell-steps count each
 * job's interior cells times the steps of the work items that computed them; the
 * skipped ones are those of items whose region had nothing burning (discrete), b = 0
 * (differentiable forward) or a = 0 (adjoint), which change nothing and are not
 * computed. ms_forward / ms_adjoint: device time of the persistent forward / adjoint
 * kernels (CUDA events in the submission's graph); ms_kernels_from_start: from the
 * start of the graph to the end of the last of them (initial states, prep, both
 * kernels). These count the queued jobs only; direct_jobs ran through contexts of their
 * own, with direct_cell_steps (H W T, twice for an adjoint) in ms_direct (CUDA events
 * around them, context set-up included). The paper has no counterpart: reporting for
 * the batch's roofline. */
typedef struct pf_batch_stats_t {
    long long disc_cell_steps, disc_skipped;
    long long diff_cell_steps, diff_skipped;
    long long adj_cell_steps, adj_skipped;
    double ms_forward, ms_adjoint, ms_kernels_from_start;
    int waves;
    int direct_jobs;
    long long direct_cell_steps;
    double ms_direct;
} pf_batch_stats_t;
int pf_batch_last_stats(pf_batch_stats_t* out);

/* Message of the last failure on ctx (or of the last context-free call when ctx is
 * NULL). Never NULL; valid until the next call on the same context. */
const char* pf_last_error(const pf_ctx* ctx);

/* Library version string. */
const char* pf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PFIRE_H */
