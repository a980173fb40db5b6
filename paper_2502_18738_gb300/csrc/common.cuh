// Internal declarations shared by the libpfire translation units (not installed).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tma.cuh"

namespace pf {

// f_p(x) = tanh(C x) (Eq. 5/8), the paper's constant rounded to FP32.
constexpr float kC = 1.1486328125f;

// Neighbour offsets (dr, dc) from the receiving cell to the burning neighbour, fixed
// direction order d = 0..7.
__host__ __device__ constexpr int dir_dr(int d) { return d < 3 ? -1 : (d < 5 ? 0 : 1); }
__host__ __device__ constexpr int dir_dc(int d) {
    return (d == 0 || d == 3 || d == 5) ? -1 : ((d == 1 || d == 6) ? 0 : 1);
}

// Pitched layouts: every internal per-cell plane has H rows of `pitch` elements,
// pitch = W rounded up to 16 (16-byte rows for uint8, 64-byte rows for FP32), so that
// rows are valid TMA strides and 16-byte vector accesses. Columns [W, pitch) hold the
// neutral value (state 0 / a = b = q = 0) and behave as cells outside the grid.
inline int pitch_of(int W) { return (W + 15) & ~15; }

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon et al., SC'11): per round, the two multipliers act on words 0
// and 2; their high halves are xored with the odd words and the key; the key advances
// by the two Weyl increments between rounds.
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                       uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return {c0, c1, c2, c3};
}

// Uniform in [0, 1) from the top 24 bits: exact in FP32.
__device__ __forceinline__ float u24(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

// Byte-lane helpers for uint8 states packed 4 per 32-bit word (states are 0..3, so
// only bits 0-1 of each byte are ever set).
__device__ __forceinline__ uint32_t lanes_eq2(uint32_t x) { return (x >> 1) & ~x & 0x01010101u; }
__device__ __forceinline__ uint32_t lanes_eq1(uint32_t x) { return x & ~(x >> 1) & 0x01010101u; }

// Continuous-state encoding of a = P[ever ignited]: A = a when a < 1/2, A = -(1 - a)
// otherwise (the sign bit selects the complement; -0.0 is a = 1). FP32 keeps both a
// near 0 and 1 - a near 0 accurate this way, which the update n = (1 - a) P needs in
// cells that have almost surely ignited.
__device__ __forceinline__ void a_decode(float A, float& a, float& ua) {
    if (signbit(A)) { a = 1.0f + A; ua = -A; } else { a = A; ua = 1.0f - A; }
}
__device__ __forceinline__ float a_encode(float a, float ua) { return a < 0.5f ? a : -ua; }

// ------------------------------------------------------ extended-range (tiered) state
// Ahead of a fire the mean-field state falls far below FP32's range (2^-149): values of
// a and b decay by a roughly constant factor per cell towards the light cone, and the
// front, a pulled front, moves at a speed set by how deep that leading edge is carried.
// Truncating it at FP32's floor slows the front measurably within a few hundred steps;
// carrying it to FP64's floor (2^-1074) does not. Cells with a < 2^-64 are therefore
// held in tiers k = 1 .. kKMax with a = A 2^(-64 k), b = B 2^(-64 k), A in [2^-64, 1):
// an FP32 mantissa with an 11-bit exponent range, below 2^-960 the cell is 0.
// Storage keeps 8 bytes per cell. A cell of tier 0 is stored as before (A complement-
// aware, B >= +0). A tiered cell stores -B (B's sign bit marks the tier) and its A
// rounded to 19 mantissa bits with k in the low 5 bits.
constexpr int kKMax = 14;  // below 2^-960 a cell is 0 (4-bit tier fields keep 15 for "a = 0")
constexpr int kKNone = 15;  // b-tier of a cell with b = 0 (and kP of a cell with no burning neighbour)
constexpr float kTierUp = 0x1p64f, kTierDown = 0x1p-64f;

// 2^(-64 d) for a tier difference 0 <= d <= 15: 1, 2^-64, and 0 from d = 2 on (a term two
// tiers down is below 2^-128 of the largest)
__device__ __forceinline__ float tier_scale(int d) { return __int_as_float(max(127 - 64 * d, 0) << 23); }

// stored (As, Bs) -> tier k and the magnitudes A, B in that tier
__device__ __forceinline__ void x_decode(float As, float Bs, float& A, float& B, int& k) {
    const uint32_t ua = __float_as_uint(As), ub = __float_as_uint(Bs);
    const bool tiered = (int32_t)ub < 0;
    k = tiered ? (int)(ua & 31u) : 0;
    A = tiered ? __uint_as_float(ua & ~31u) : As;
    B = __uint_as_float(ub & 0x7fffffffu);
}
// Per-thread tier summaries of a 4-bit-per-cell tier word (a = 0 cells hold 15, which
// belongs to no tier: such a cell computes the same under any tier's arithmetic). Fields
// of 4 bits: [0] the least tier of the word's cells (15: none), [1] the greatest (0:
// none), [2] / [3] the same for its first cell, [4] / [5] for its last cell.
__device__ __forceinline__ uint32_t tier_summary(uint32_t w) {
    uint32_t lo = 15u, hi = 0u;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const uint32_t t = (w >> (4 * m)) & 15u;
        lo = min(lo, t);
        hi = max(hi, t == 15u ? 0u : t);
    }
    const uint32_t f = w & 15u, l = w >> 28;
    return lo | (hi << 4) | (f << 8) | ((f == 15u ? 0u : f) << 12) | (l << 16) | ((l == 15u ? 0u : l) << 20);
}
__device__ __forceinline__ uint32_t ts_lo(uint32_t s) { return s & 15u; }
__device__ __forceinline__ uint32_t ts_hi(uint32_t s) { return (s >> 4) & 15u; }
__device__ __forceinline__ uint32_t ts_first_lo(uint32_t s) { return (s >> 8) & 15u; }
__device__ __forceinline__ uint32_t ts_first_hi(uint32_t s) { return (s >> 12) & 15u; }
__device__ __forceinline__ uint32_t ts_last_lo(uint32_t s) { return (s >> 16) & 15u; }
__device__ __forceinline__ uint32_t ts_last_hi(uint32_t s) { return (s >> 20) & 15u; }

// The window of a thread owning the 8-cell column strip at (strip, x) of a 64 x 64 region
// (rows ys-1 .. ys+8, columns x-1 .. x+1) from the summaries of its own strip (c), the
// neighbouring columns (at -dl / +dr) and the strips above and below: whether its cells
// that are not 0 are all in one tier, and that tier (k0 = 0 when all are 0).
__device__ __forceinline__ bool window_one_tier(const uint32_t* sum, int tid, int dl, int dr, bool above,
                                                bool below, int row_stride, uint32_t c, uint32_t& k0) {
    const uint32_t l = sum[tid - dl], r = sum[tid + dr];
    uint32_t lo = min(min(ts_lo(c), ts_lo(l)), ts_lo(r));
    uint32_t hi = max(max(ts_hi(c), ts_hi(l)), ts_hi(r));
    if (above) {
        const uint32_t* a = sum + tid - row_stride;
        lo = min(min(lo, ts_last_lo(a[0])), min(ts_last_lo(a[-dl]), ts_last_lo(a[dr])));
        hi = max(max(hi, ts_last_hi(a[0])), max(ts_last_hi(a[-dl]), ts_last_hi(a[dr])));
    }
    if (below) {
        const uint32_t* b = sum + tid + row_stride;
        lo = min(min(lo, ts_first_lo(b[0])), min(ts_first_lo(b[-dl]), ts_first_lo(b[dr])));
        hi = max(max(hi, ts_first_hi(b[0])), max(ts_first_hi(b[-dl]), ts_first_hi(b[dr])));
    }
    k0 = lo == 15u ? 0u : lo;
    return lo >= hi;
}

// the tier of a stored cell (0 for tier 0 and for a = 0)
__device__ __forceinline__ int x_tier(float As, float Bs) {
    return (int32_t)__float_as_uint(Bs) < 0 ? (int)(__float_as_uint(As) & 31u) : 0;
}
// A of a tiered cell as it is kept: 19 mantissa bits (round to nearest)
__device__ __forceinline__ float x_round19(float A) { return __uint_as_float((__float_as_uint(A) + 0x10u) & ~31u); }
__device__ __forceinline__ void x_encode(float A, float B, int k, float& As, float& Bs) {
    if (k == 0) {
        As = A;
        Bs = B;
    } else {
        As = __uint_as_float((__float_as_uint(A) & ~31u) | (uint32_t)k);  // A already rounded
        Bs = __uint_as_float(__float_as_uint(B) | 0x80000000u);
    }
}
// Keep a non-complement cell normalised after its update: A in [2^-64, 1) for k >= 1
// (A rounded to 19 bits there), and a cell below the deepest tier becomes 0. A cell that
// is already normalised is left exactly as it is, so a cell whose inputs do not change
// does not change either (which makes skipping quiescent tiles exact).
__device__ __forceinline__ void x_renorm(float& A, float& B, int& k) {
    if (!(A > 0.0f)) {  // complement-encoded (a >= 1/2, tier 0) or exactly 0
        if (__float_as_uint(A) == 0u) { B = 0.0f; k = 0; }
        return;
    }
    if (A >= 1.0f && k >= 1) { A *= kTierDown; B *= kTierDown; --k; }
    while (A < kTierDown) {
        if (k == kKMax) { A = 0.0f; B = 0.0f; k = 0; return; }
        A *= kTierUp; B *= kTierUp; ++k;
    }
    if (k > 0) {
        A = x_round19(A);
        if (A >= 1.0f) { A *= kTierDown; B *= kTierDown; --k; }  // rounded up to 1: exact 2^-64 a tier up
    }
}

// The cell's own part of a differentiable step in the tiered arithmetic, from the P and S
// accumulated over its neighbours at tier kP (kKNone: no burning neighbour): A, B, k are
// the cell's own (A complement-encoded when k = 0 and a >= 1/2); returns A', B', k' (A'
// rounded when tiered). The update runs at tier min(k, kP) and renormalises.
__device__ __forceinline__ void x_own(float P, float S, int kP, float A, float B, int k, float pc, float& An,
                                      float& Bn, int& kn) {
    if (signbit(A)) {  // a >= 1/2, tier 0
        const float a = __fadd_rn(1.0f, A), ua = -A;
        const float n = __fmul_rn(__fmul_rn(ua, P), tier_scale(kP));
        An = a_encode(__fadd_rn(a, n), __fmul_rn(ua, S));
        Bn = fmaf(pc, B, n);
        kn = 0;
        return;
    }
    const int s = __float_as_uint(A) == 0u ? kP : min(k, kP);
    const float h = tier_scale(max(k - s, 0));  // a = 0 (s = kP may exceed k): A = B = 0, h unused
    const float as = __fmul_rn(A, h), bs = __fmul_rn(B, h);
    const float ua = k == 0 ? __fsub_rn(1.0f, A) : 1.0f;
    const float n = __fmul_rn(ua, __fmul_rn(P, tier_scale(kP - s)));
    const float an = __fadd_rn(as, n);
    Bn = fmaf(pc, bs, n);
    An = s == 0 ? a_encode(an, __fmul_rn(ua, S)) : an;
    kn = s;
    x_renorm(An, Bn, kn);
}

// One cell's differentiable step in the tiered arithmetic (the definition every kernel
// follows; on tier-0 inputs it is the plain FP32 update below, bit for bit).
//   nb[d], nk[d]: the neighbours' B magnitudes and tiers (B = 0 outside the grid);
//   q[d]: the folded factors into this cell; A, B, k: the cell's own.
// P is accumulated at the tier kP of the largest contributions, the least tier of the
// neighbours with b > 0 (terms two or more tiers down vanish); when kP >= 1 every true
// term is below 2^-61, so the survival product stays 1 and P is a plain sum.
__device__ __forceinline__ void x_update(const float (&nb)[8], const int (&nk)[8], const float (&q)[8], float A,
                                         float B, int k, float pc, float& An, float& Bn, int& kn) {
    int kP = kKNone;
#pragma unroll
    for (int d = 0; d < 8; ++d) kP = min(kP, nb[d] != 0.0f ? nk[d] : kKNone);
    const bool kP0 = kP == 0;
    float P = 0.0f, S = 1.0f;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const float x = __fmul_rn(__fmul_rn(nb[d], q[d]), tier_scale((nb[d] != 0.0f ? nk[d] : kKNone) - kP));
        P = fmaf(x, S, P);
        S = kP0 ? fmaf(-x, S, S) : S;
    }
    x_own(P, S, kP, A, B, k, pc, An, Bn, kn);
}

// The same update when the cell and every neighbour are in tier 0, from the P and S that
// ign_acc accumulated over x_d = b_i q_dj (rounded products): the same roundings as
// x_update on such inputs (every tier factor there is an exact 1).
__device__ __forceinline__ void x_update_t0(float P, float S, float A, float B, float pc, float& An, float& Bn,
                                            int& kn) {
    float a, ua;
    if (signbit(A)) {
        a = __fadd_rn(1.0f, A);
        ua = -A;
    } else {
        a = A;
        ua = __fsub_rn(1.0f, A);
    }
    const float n = __fmul_rn(ua, P);
    An = a_encode(__fadd_rn(a, n), __fmul_rn(ua, S));
    Bn = fmaf(pc, B, n);
    kn = 0;
    if (!signbit(A)) x_renorm(An, Bn, kn);
}

// Scaled-adjoint exponent of a cell (see the scaled adjoint below): its tier, 0 for
// a >= 1/2, and 255 (kSigmaZero) for a == 0.
__device__ __forceinline__ int x_sigma(float As, float Bs) {
    const uint32_t ua = __float_as_uint(As);
    if (ua == 0u) return 255;  // a == 0 (kSigmaZero)
    return x_tier(As, Bs);
}
// 2^e for an integer exponent, 0 below 2^-126 (terms scaled that far down are dropped)
__device__ __forceinline__ float exp2i(int e) {
    e = min(e, 127);
    return e < -126 ? 0.0f : __int_as_float((e + 127) << 23);
}

// Eq. 9 over the factors x_d = b_i q_dj of a differentiable step: S = prod_d (1 - x_d)
// and P = 1 - S, accumulated as P += x_d S (the term x_d prod_{e<d} (1 - x_e)). Both are
// sums / products of non-negative terms, so P keeps its relative accuracy when it is
// small and S when P is close to 1.
__device__ __forceinline__ void ign_acc(float x, float& P, float& S) {
    P = fmaf(x, S, P);
    S = fmaf(-x, S, S);
}

// Scaled adjoint. Ahead of the fire the exact lambda grows about 4x per step backwards
// in time while the states it multiplies shrink as fast; their products, which carry
// the (pulled) front's sensitivity, stay O(1), but lambda itself overflows FP32 within
// ~60 steps (and FP64 within a few hundred). The adjoint therefore stores
// mu_j = lambda_j 2^(-64 sigma_j) with sigma_j the tier of the cell's own state (x_sigma;
// lambda ~ 1 / a spans 2^64 within a tier, well inside FP32), and rescales a transfer
// between cells of different tiers by the exact power of two 2^(64 (sigma_j - sigma_i)).
// Within one tier nothing is rescaled. sigma = kSigmaZero marks a == 0 exactly (outside
// the light cone, or non-burnable): there lambda multiplies only exact zeros and is held
// at 0.
constexpr int kSigmaZero = 255;

// ---------------------------------------------------------------- launchers
struct PrepArgs {
    int H, W, pitch;
    const float *E, *pveg, *pden, *V, *th;  // dense H*W, nullable
    const uint8_t* burnable;                 // dense H*W, nullable
    const float* slope;                      // dense [H][W][3][3] degrees (replaces E), nullable
    float p_h, c1, c2, a, l;
    // reach mask (nullable, prep only): q is computed in the 32 x 32 cell blocks whose
    // byte reach[(r / 32) * reach_bw + c / 32] is set and left as it is elsewhere
    const uint8_t* reach;
    int reach_bw;
    // dL/dq tiles (nullable, prep adjoint only): dL/dq can be nonzero only in the 48 x 48
    // tiles whose byte gq_dirty[(r / 48) * gq_tiles_x + c / 48] is set
    const uint8_t* gq_dirty;
    int gq_tiles_x;
    // derived on the host in FP64 and split into hi + lo floats:
    // a * 180/pi, 1/l and 1/(sqrt(2) l)
    float adeg_hi, adeg_lo, ikl_e_hi, ikl_e_lo, ikl_d_hi, ikl_d_lo;
};
// fill the derived hi/lo fields of PrepArgs from p_h, c1, c2, a, l
void prep_derive(PrepArgs& g);

void launch_prep(const PrepArgs& g, float* q, cudaStream_t s);
// Reach mask of a differentiable state ab ([2][H][pitch], encoded a then b) over 32 x 32
// cell blocks (ceil(H/32) x ceil(W/32) bytes, row-major): reach[B] = 1 iff a block within
// Chebyshev block distance `radius` of B holds a cell with a > 0 or b > 0. tmp: scratch
// of the same size.
int prep_reach_bytes(int H, int W);
void launch_prep_reach(const float* ab, int H, int W, int pitch, int radius, uint8_t* tmp, uint8_t* reach,
                       cudaStream_t s);
// acc |= in over nb mask bytes (the union of two reach masks)
void launch_reach_or(uint8_t* acc, const uint8_t* in, int nb, cudaStream_t s);
// dL/dq -> per-block FP64 partials of dL/d(p_h, c1, c2, a) (partials[nblk][4]) and
// accumulation of per-cell gradients (dense H*W, nullable). Gq is left all zeros.
int prep_adjoint_blocks(int H, int W);
void launch_prep_adjoint(const PrepArgs& g, float* Gq, double* partials, float* gpveg,
                         float* gpden, cudaStream_t s);
// acc[0..3] += fixed-order FP64 sum of partials[nblk][4]
void launch_reduce_partials(const double* partials, int nblk, double* acc, cudaStream_t s);

struct DiscreteArgs {
    int H, W, pitch, R;
    float p_continue;
    uint32_t key0, key1, fire, run0;
    // accumulator (nullable): dense [R][H][W] FP32; a cell that ignites gets the p_ignite
    // it ignited with. Kernels write it for cells in rows [acc_r0, acc_r1) and columns
    // [acc_c0, acc_c1) of the grid they compute exactly once (the launcher sets these).
    float* acc;
    int acc_r0, acc_r1, acc_c0, acc_c1;
    // near-tie counters (nullable): [0] cells whose ignition draw lies within kNearTie of
    // p_ignite, [1] burning cells whose continue draw lies within kNearTie of p_continue;
    // counted for the cells in the same rows / columns as the accumulator
    unsigned long long* ties;
};
constexpr float kNearTie = 1e-6f;
void launch_discrete_step(const DiscreteArgs& g, const uint8_t* S, uint8_t* Sn, const float* q,
                          uint32_t step, cudaStream_t s);
// DCA gradient of one step (the paper's accumulator path): for each cell j that ignites
// between S (step t) and Sn (t + 1) in any realisation, Gq[d][j] += w_j beta_i
// prod_{e != d} (1 - beta_e q_ej), beta the burning indicators of S; w dense [R][H][W]
// (dL/dacc); realisations are summed in a fixed order.
void launch_dca_step(const DiscreteArgs& g, const uint8_t* S, const uint8_t* Sn, const float* q, const float* w,
                     float* Gq, cudaStream_t s);
// temporal-blocked: k <= KH steps per launch from global step `step`; `tin` is a 3-D
// tensor map over the [R][H][pitch] uint8 input buffer with box {160, TH + 2 KH, 1}.
// skipped (nullable) accumulates the interior cell-steps of tiles with nothing burning.
int discrete_blocked_tile_rows();
int discrete_blocked_max_k();  // steps per launch the column halo supports
size_t discrete_blocked_smem(int TH, int KH);
// pa: NULL = q read from q; else q recomputed in the kernel from pa's fields (q unused)
void launch_discrete_blocked_impl(const DiscreteArgs& g, const CUtensorMap* tin, int TH, int KH, uint8_t* Sn,
                                  const float* q, const PrepArgs* pa, uint32_t step, int k, int* err, TmaHook hk,
                                  unsigned long long* skipped, cudaStream_t s);

void launch_diff_step(int H, int W, int pitch, float p_continue, const float* ab, float* ab_next,
                      const float* q, cudaStream_t s);
// the same steps with q recomputed in the kernel from the fields of PrepArgs (prep's
// arithmetic) instead of read from materialised planes
void launch_diff_step_rc(const PrepArgs& g, float p_continue, const float* ab, float* ab_next, cudaStream_t s);
void launch_discrete_step_rc(const DiscreteArgs& g, const uint8_t* S, uint8_t* Sn, const PrepArgs& pa, uint32_t step,
                             cudaStream_t s);
// temporal-blocked differentiable forward: n <= diff_blocked_halo() steps per launch.
// tab: 3-D map over the input (A, b) buffer (pitch, H, 2), box {64, 64, 2};
// tq: 3-D map over q (pitch, H, 8), box {64, 64, 8}. out (nullable) receives the state
// after n steps; all_out (nullable) receives the state after each step s at
// all_out + s * all_stride.
int diff_blocked_halo();
int diff_blocked_box_rows();
int diff_blocked_box_cols();
int diff_blocked_configure();
// halo: 8, or 4 when every launch of the chain has n <= 4 (fixes the tile geometry).
// Only the tiles listed by the pre-pass launch_fwd_tiles run; it decides from the tile
// activity act_in (b > 0 in a tile's interior, from the previous launch's act_out or from
// launch_fwd_act_init at the start of a chain) and handles the quiescent tiles itself.
// k_diff_blocked writes act_out for the tiles it runs. skipped (nullable) accumulates the
// interior cell-steps of quiescent tiles. tile_count: two device ints, the count and the
// kernel's work counter (its CTAs take tiles dynamically), both zeroed by the pre-pass.
int diff_blocked_tiles(int halo, int H, int pitch);
void launch_fwd_act_init(int halo, const float* ab, int H, int pitch, uint8_t* act, uint8_t* qrun,
                         cudaStream_t s);
// The same from the act_out an earlier chain recorded for the state (same halo).
void launch_fwd_act_seed(int halo, const uint8_t* seed, int H, int pitch, uint8_t* act, uint8_t* qrun,
                         cudaStream_t s);
// qrun: per tile, the number of consecutive launches of the chain it has been quiescent
// in (saturating at 255); out_age > 0: out holds the input state of the launch out_age
// launches back, so tiles with qrun >= out_age need no copy into it (0: out holds nothing).
// seg_rng (nullable): all_out lies in a segment buffer reused across segments, whose
// slots zero_base + s * all_stride (s < zero_slots) hold zeros for each tile outside its
// dirty slot range seg_rng[tile] = lo | hi << 16 ([lo, hi), empty when lo >= hi); void
// tiles (a = b = 0 in the whole region) write nothing but zeros into the launch's own
// slots where they are dirty (see k_fwd_tiles).
// frozen (segment buffers only, launches aligned with the adjoint's): quiescent tiles get
// kFrozen in act_out, and those with b = 0 in the 5 x 5 interiors around them write only
// the launch's last slot (the next launch's input): every tile whose region reaches into
// them is frozen too and reads its first slot instead of the intermediate ones. With
// slot0 (the segment's first state, slot 0 of the buffer) as well, those with b = 0 in
// the 7 x 7 interiors and no change since slot 0 in the 5 x 5 write nothing (kStale; see
// k_fwd_tiles).
// out_dirty (nullable, with out a checkpoint slot): per tile of this geometry, whether the
// slot's interior may hold nonzeros; all-zero tiles (a = 0) are written only where it is
// set (all tiles if dirty_unknown), and it is updated to the state written.
// written (nullable) accumulates the cells the pre-pass copied or zero-filled.
// Returns false (nothing launched) when all_out's slots fall outside the segment buffer.
bool launch_fwd_tiles(int halo, const float* in, int H, int W, int pitch, int n, const uint8_t* act_in,
                      uint8_t* act_out, uint8_t* qrun, int* tile_list, int* tile_count, float* out,
                      int out_age, float* all_out, size_t all_stride, uint32_t* seg_rng, const float* slot0,
                      float* zero_base, int zero_slots, bool frozen, uint8_t* out_dirty, bool dirty_unknown,
                      unsigned long long* skipped, unsigned long long* written, cudaStream_t s);
// Tile tape of a taped forward: the interior states of every listed (live) tile of a
// blocked launch, kept so that the adjoint's segment recompute can copy them instead of
// computing them again. A block is one state of one tile's interior, [2][kI][kI] FP32
// (kI = the interior side), stored as the launch writes its slots (x_encode form). The
// blocks of a launch are base + li * n + s (li: the tile's index in the launch's list,
// s: its step); `used` (device) is the number of blocks taken so far.
struct TileTape {
    float* data;                        // NULL: no tape
    unsigned long long* used;
    unsigned long long cap;             // blocks
};
// pa: NULL = q staged from the planes of tq; else q recomputed in the kernel from pa's fields
// tape (data NULL: none): the launch's live tiles' states are also written as blocks
void launch_diff_blocked(int halo, const CUtensorMap* tab, const CUtensorMap* tq, const PrepArgs* pa, int H, int W,
                         int pitch, float pc, int n, const int* tile_list, int* tile_count, float* out, float* all_out,
                         size_t all_stride, uint8_t* act_out, unsigned long long* skipped, int nsm, int* err,
                         TmaHook hk, TileTape tape, cudaStream_t s);
// After a taped launch: meta[4 L ..] = {base, n, count, ok} of launch record L (ok: every
// block fitted), the list copied to lists + L * list_cap, and tape.used advanced.
void launch_tape_record(TileTape tape, const int* tile_count, const int* tile_list, int n, int L,
                        unsigned long long* meta, int* lists, int list_cap, cudaStream_t s);
// A segment recompute launch of n steps from the tape instead of k_diff_blocked: for every
// tile of the recompute's list, its n states from the blocks of record {base, n_rec,
// count} (inv: tile -> index in the record's list, built here from rec_list) into
// all_out's slots, and its activity after the launch into act_out (kQb kept), as
// k_diff_blocked writes them. A listed tile missing from the record adds to *missing.
// nsm: the device's SM count (the grid is eight blocks an SM).
void launch_tape_unpack(int halo, const float* tape_data, unsigned long long base, int n_rec, int rec_count,
                        const int* rec_list, int* inv, int ntiles, const int* tile_list, const int* tile_count,
                        int n, int H, int pitch, float* all_out, size_t all_stride, uint8_t* act_out, int* missing,
                        int nsm, cudaStream_t s);
// lam: scaled adjoint (mu_a, mu_b) [2][H][pitch]; sig: its exponents uint8 [H][pitch]
void launch_adjoint_step(int H, int W, int pitch, float p_continue, const float* ab, const float* q,
                         const float* lam1, const uint8_t* sig1, float* lam0, uint8_t* sig0, float* Gq,
                         cudaStream_t s);
// terminal scaled adjoint from dL/da_T, dL/db_T (dense, nullable) and the state at T
void launch_adjoint_init(const float* dLda, const float* dLdb, const float* ab, int H, int W, int pitch,
                         float* lam, uint8_t* sig, cudaStream_t s);
// Tile activity flags of the blocked forward (one byte per 48 x 48 interior tile, the
// tiles of the 8-cell-halo geometry): b > 0 / a > 0 somewhere in the tile's interior.
constexpr uint8_t kActB = 1, kActA = 2;
// recorded per launch of an aligned recompute (see k_fwd_tiles): b = 0 in the 3 x 3
// interiors around the tile at the launch's first state, so the tile's region is
// constant over the launch's steps
constexpr uint8_t kFrozen = 4;
// Segment recompute (aligned launches): kQb: the tile was quiescent in every launch of the
// segment before this one (its state at the launch's input is the segment's first state,
// slot 0); kQt: ... and in this one too; kStale: the tile's state is not in this launch's
// last slot (it skipped the write; see k_fwd_tiles).
constexpr uint8_t kQb = 8, kQt = 16, kStale = 32;
// an adjoint tile-list entry with this bit reads the state of its launch's first step
// for every step (its region is constant over the launch); with kTileCkptBit as well it
// reads it from slot 0, the segment's first state (the 3 x 3 tiles around it are kQb)
constexpr int kTileFrozenBit = 1 << 30;
constexpr int kTileCkptBit = 1 << 29;
constexpr int kTileIndexMask = kTileCkptBit - 1;

// Adds a block's per-thread counts to a per-launch counter with one global atomic per
// block (every tile of a launch would otherwise hit the same address). s: a __shared__
// word zeroed before a __syncthreads that precedes the call; every thread of the block
// calls this.
__device__ __forceinline__ void block_count(unsigned long long* g, unsigned long long& s, unsigned long long v) {
    if (v) atomicAdd(&s, v);
    __syncthreads();
    if (threadIdx.x == 0 && g && s) atomicAdd(g, s);
}

// temporal-blocked adjoint with TMEM working set: n <= adjoint_blocked_max_steps() steps
// t = t1-1 .. t1-n per launch. tst: 3-D map over a buffer of consecutive states
// (pitch, H, 2 * nstates), box {64, 64, 2}; the state at t1-1-m is state index zlast-m,
// except state index 0, which is read through tst0 (a map of one state, the same box:
// a checkpoint that is not copied into the buffer, or tst itself).
// tq as for launch_diff_blocked. Gq is accumulated. Only the tiles listed by the
// pre-pass launch_adjoint_tiles run: from A_latest, the encoded a plane of the state at
// t1-1, it lists the tiles with a > 0 somewhere in their region (tile_list, capacity
// adjoint_blocked_tiles(); tile_count: three device ints zeroed by the pre-pass: the
// count listed from the front, the kernel's work counter, the count listed from the back
// (frozen tiles)) and writes lambda = 0,
// sigma = kSigmaZero for the others, whose interior cell-steps it adds to skipped.
int adjoint_blocked_max_steps();
int adjoint_blocked_configure();
int adjoint_blocked_tiles(int H, int pitch);
void launch_adjoint_tiles(const float* A_latest, int H, int W, int pitch, int n, float* lam_out, uint8_t* sig_out,
                          int* tile_list, int* tile_count, uint8_t* gq_dirty, unsigned long long* skipped,
                          cudaStream_t s);
// The same pre-pass from the forward's tile activity at a state s >= t1 - 1 (a never
// decreases, so a tile with kActA in none of the 3 x 3 interiors around it has a = 0 in
// its region at t1 - 1) instead of the state itself; a quiescent tile's lambda and sigma
// are written only until both ping-pong buffers hold them (deadcnt[tile] counts that).
// use_frozen: the flags come from a recompute launch aligned with this adjoint launch;
// tiles recorded kFrozen are listed with kTileFrozenBit (their interior cell-steps are
// added to frozen_steps, nullable).
// Both pre-passes set gq_dirty[tile] (nullable) for every listed tile that may add to dL/dq
// (the frozen ones add nothing).
void launch_adjoint_tiles_flags(const uint8_t* act, int H, int W, int pitch, int n, float* lam_out, uint8_t* sig_out,
                                uint8_t* deadcnt, int* tile_list, int* tile_count, bool use_frozen,
                                uint8_t* gq_dirty, unsigned long long* skipped, unsigned long long* frozen_steps,
                                cudaStream_t s);
// The listed non-frozen tiles run in k_adjoint_blocked (frozen_only false); the frozen ones
// (listed from the back) in k_adjoint_frozen (frozen_only true), which stages q, the state
// and lambda_in (tlam: a map of lam_in's two planes, the same box) by TMA. A launch of the
// blocked adjoint is both calls. tile_count: [0] front count, [1] k_adjoint_blocked's work
// counter, [2] frozen count, [3] k_adjoint_frozen's work counter (zeroed by the pre-passes).
void launch_adjoint_blocked(const CUtensorMap* tst, const CUtensorMap* tst0, const CUtensorMap* tq,
                            const CUtensorMap* tlam, int H, int pitch, float pc, int zlast, int n,
                            const float* lam_in, const uint8_t* sig_in, float* lam_out, uint8_t* sig_out, float* Gq,
                            const int* tile_list, int* tile_count, int nsm, int* err, TmaHook hk, bool frozen_only,
                            cudaStream_t s);
void launch_ignition_map_discrete(const DiscreteArgs& g, const uint8_t* S, const float* q, float* P,
                                  cudaStream_t s);
void launch_ignition_map_diff(int H, int W, int pitch, const float* ab, const float* q, float* P,
                              cudaStream_t s);
// dense FP32 (a, b) [2][H][W]  <->  pitched encoded (A, b) [2][H][pitch]
void launch_diff_pack(const float* dense, int H, int W, int pitch, float* ab, cudaStream_t s);
void launch_diff_unpack(const float* ab, int H, int W, int pitch, float* dense, cudaStream_t s);

// batched fires (kernels_batch.cu)
struct BatchJobDev {
    int H, W, P, T, form, nblk, tiles_x, tiles_y;
    uint32_t key0, key1, run, fire;
    float pc;
    void* st[2];
    const float* q;
    int* gen;
    void* out;
    // differentiable jobs with an adjoint: every state [T+1][2][H][P] (the forward writes
    // it), the scaled adjoint ping-pong at block boundaries and dL/dq [8][H][P]
    float* tape;
    float* lam[2];
    uint8_t* sig[2];
    float* Gq;
    int* gen_b;  // backward tile generations
    int btiles_x, btiles_y;
};
struct BatchPlan {
    const BatchJobDev* jobs;
    const long long* blk_start;
    const long long* tile_pref;
    const int* jobs_in_blk;
    int max_blk;
    long long total;
    unsigned long long* counter;
    int* err;
    long long wait_limit_ns;  // bound on one wait for a neighbouring tile
    int withhold;
    // nullable: interior cell-steps of the items that were stepped / skipped (nothing
    // burning, or a = 0 for the adjoint, in the item's region), indexed by BatchStat
    unsigned long long* stats;
};
enum BatchStat { kStatDisc, kStatDiscSkip, kStatDiff, kStatDiffSkip, kStatAdj, kStatAdjSkip, kStatCount };
int batch_tile_rows();
int batch_tile_cols();
int batch_steps_per_item();
int batch_blocks_per_sm();
void launch_batch(const BatchPlan& plan, int grid, cudaStream_t s);
// reverse-time adjoint of the differentiable jobs with a tape: plan items are (job,
// backward tile, block counted from the job's last block)
int batch_adj_tile_rows();
int batch_adj_tile_cols();
int batch_adj_blocks_per_sm();
int batch_adj_configure();
void launch_batch_adj(const BatchPlan& plan, int grid, cudaStream_t s);

}  // namespace pf
