// Temporal-blocked reverse-time adjoint of the differentiable step (the same update
// as k_adjoint_step, n <= 7 steps per launch), with the per-cell working set in TMEM.
//
// Persistent kernel, one CTA (512 threads) per SM, 48 x 48 interior tiles staged as
// 64 x 64 regions (8-cell halo). For each tile the CTA
//   * moves the region's q planes (TMA-staged, prefetched during the previous tile) into
//     tensor memory, and zeroes a dL/dq accumulator there: each thread owns an 8-cell
//     column strip and 128 TMEM columns of its warp's lane quarter (8 q + 8 dL/dq per cell);
//   * keeps lambda = dL/d(a, b) of its cells in registers;
//   * for each of the n steps t = t1-1 .. t0 streams the recomputed state (A, b) at t
//     through a double-buffered TMA stage, and
//       - per target cell j: P_j, the leave-one-out products of the 8 factors
//         (1 - b_i q_dj) by prefix / suffix products, l_P_j = (l_a'_j + l_b'_j)(1 - a_j),
//         l_a_j = l_a'_j - l_n_j P_j, dL/dq_dj += l_P_j b_i LOO_dj, and the 8 contributions
//         C_dj = l_P_j q_dj LOO_dj to the sources i = j + d;
//       - gathers l_b_i = p_c l_b'_i + sum of the C arriving at i: within a thread's
//         strip directly, across lanes by warp shuffles, across warps and strips through
//         small double-buffered shared-memory exchange rows (no atomics, fixed order);
//   * carries lambda in the scaled form of common.cuh (per-cell power-of-two exponents
//     from the cell's own state, so it stays finite ahead of the fire);
//   * writes lambda at t0 for the interior and adds the tile's dL/dq into global memory.
// The halo shrinks by one cell per step, so the 48 x 48 interior is exact for n <= 7.
// Tiles whose region is constant over the launch (frozen) run in k_adjoint_frozen below.
#include <cuda.h>

#include <cstddef>
#include <type_traits>

#include "common.cuh"
#include "tma.cuh"
#include "tmem.cuh"

namespace pf {

namespace {

constexpr int kRT = 64, kCT = 64;
constexpr int kHalo = 8;
constexpr int kIR = kRT - 2 * kHalo, kIC = kCT - 2 * kHalo;
constexpr int kM = 8;
constexpr int kStrips = kRT / kM;
constexpr int kThreads = kCT * kStrips;  // 512
constexpr int kPlane = kRT * kCT;
constexpr int kMaxSteps = kHalo - 1;
constexpr uint32_t kTmemCols = 512;

struct Smem {
    float q[8 * kPlane];                 // q stage of the next tile (TMA)
    float st[2][2 * kPlane];             // state stages (A, b), double buffered (TMA)
    float vtop[2][kStrips][3][kCT];      // [parity][strip][dc+1][col]: C for row ys-1
    float vbot[2][kStrips][3][kCT];      // C for row ys+8
    float el2r[2][kStrips][kM];          // x = 31 -> x = 32 (dc = +1), rows of the strip
    float er2l[2][kStrips][kM];          // x = 32 -> x = 31 (dc = -1)
    float edump[kThreads];               // where the other threads' exchange stores go
    uint32_t ks[2][kThreads];            // tier summaries at t of each thread's 8 cells, by step parity
};
static_assert(offsetof(Smem, el2r) % 16 == 0 && offsetof(Smem, er2l) % 16 == 0, "16-byte loads of the exchange rows");

__device__ __forceinline__ void origin(int tile, int tiles_x, int& r0, int& c0) {
    r0 = (tile / tiles_x) * kIR - kHalo;
    c0 = (tile % tiles_x) * kIC - kHalo;
}

__global__ void __launch_bounds__(kThreads, 1)
    k_adjoint_blocked(const __grid_constant__ CUtensorMap tst, const __grid_constant__ CUtensorMap tst0,
                      const __grid_constant__ CUtensorMap tq, int H,
                      int pitch, float pc, int zlast, int n, int tiles_x, const int* __restrict__ tiles,
                      const int* __restrict__ ntiles_live, int* __restrict__ next,
                      const float* __restrict__ lam_in, const uint8_t* __restrict__ sig_in,
                      float* __restrict__ lam_out, uint8_t* __restrict__ sig_out, float* __restrict__ Gq,
                      int* __restrict__ err, TmaHook hk) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    __shared__ __align__(8) uint64_t sbar[2];
    __shared__ __align__(8) uint64_t qbar;
    __shared__ uint32_t tslot;
    // list entries of this CTA's tiles l = 0, 1, ... at tring[l & 3] (-1: no more). Tiles
    // are handed out dynamically: the first is tiles[blockIdx.x], each next one comes from
    // the work counter next (claimed by thread 0 one tile ahead of its use, two when a
    // launch has fewer than 3 steps, so the TMA prefetch of its q and first states keeps
    // its distance).
    __shared__ int tring[4];

    const int tid = threadIdx.x;
    const int x = tid % kCT;
    const int strip = tid / kCT;
    const int ys = strip * kM;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const size_t gplane = (size_t)H * pitch;
    // the live tiles of the pre-pass's list, from its front (the frozen ones, stored from
    // its back and counted in ntiles_live[2], run in k_adjoint_frozen)
    const int ntiles = ntiles_live[0];
    if ((int)blockIdx.x >= ntiles) return;
    // thread 0's queue state, in shared memory to keep it out of the hot loop's registers:
    // entries of tiles 0 .. qstate[0]-1 are in tring; qstate[1]: no more tiles
    // (and the list's front count and capacity)
    __shared__ int qstate[4];
    if (tid == 0) {
        qstate[0] = qstate[1] = 0;
        qstate[2] = ntiles_live[0];
        qstate[3] = tiles_x * ((H + kIR - 1) / kIR);
    }
    auto ensure = [&](int l) {  // thread 0: make the entry of tile l known
        while (qstate[0] <= l) {
            const int f = qstate[0];
            int e = -1;
            if (!qstate[1]) {
                const int k = f == 0 ? (int)blockIdx.x : (int)gridDim.x + atomicAdd(next, 1);
                if (k < qstate[2]) e = tiles[k];
                else qstate[1] = 1;
            }
            tring[f & 3] = e;
            qstate[0] = f + 1;
        }
    };

    if (tid == 0) {
        mbar_init(&sbar[0], 1);
        mbar_init(&sbar[1], 1);
        mbar_init(&qbar, 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&tslot, kTmemCols);
    tmem_sync_threads();
    // this thread's TMEM columns: lane quarter warp % 4, column block warp / 4
    const uint32_t tbase = tslot + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * 128);

    auto issue_state = [&](int i) {  // thread 0: stage the state of local step i, if any
        const int l = i / n, m = i % n;
        ensure(l);
        const int e = tring[l & 3];
        if (e < 0) return;
        int r0, c0;
        origin(e & kTileIndexMask, tiles_x, r0, c0);
        const int s = i & 1;
        const int z = zlast - m;
        mbar_arrive_expect_tx(&sbar[s], (uint32_t)(2 * kPlane * sizeof(float)));
        if (hk.withhold) return;
        if (z == 0)
            tma_load_3d(sm.st[s], &tst0, &sbar[s], c0, r0, 0);
        else
            tma_load_3d(sm.st[s], &tst, &sbar[s], c0, r0, 2 * z);
    };
    auto issue_q = [&](int l) {  // thread 0: stage q of tile l, if any
        ensure(l);
        const int e = tring[l & 3];
        if (e < 0) return;
        int r0, c0;
        origin(e & kTileIndexMask, tiles_x, r0, c0);
        mbar_arrive_expect_tx(&qbar, (uint32_t)(8 * kPlane * sizeof(float)));
        if (!hk.withhold) tma_load_3d(sm.q, &tq, &qbar, c0, r0, 0);
    };
    if (tid == 0) {
        issue_q(0);
        issue_state(0);
        issue_state(1);
    }
    __syncthreads();  // tring[0]

    // the cross-warp exchange of a completed row: x = 31 passes its dc = +1 term to x = 32,
    // x = 32 its dc = -1 term to x = 31; every other thread stores into its own scratch
    // word, so the store is not branched on (float offsets into the shared-memory block)
    const bool ex_on = x == 31 || x == 32;
    const int ex_off = x == 31   ? (int)(offsetof(Smem, el2r) / sizeof(float)) + strip * kM
                       : x == 32 ? (int)(offsetof(Smem, er2l) / sizeof(float)) + strip * kM
                                 : (int)(offsetof(Smem, edump) / sizeof(float)) + tid;
    auto exchange = [&](int ex, int row, float right, float left) {
        reinterpret_cast<float*>(&sm)[ex_off + (ex_on ? ex * kStrips * kM + row : 0)] = x == 32 ? left : right;
    };
    // The tier summary (tier_summary) of this thread's cells in a staged state: computed
    // for step i + 1 during step i (its stage was issued a step earlier), so the
    // neighbours read it after step i's end barrier without a barrier of its own.
    auto tier_sum = [&](const float* A_, const float* B_) {
        uint32_t kword = 0u;
#pragma unroll
        for (int k = 0; k < kM; ++k) {
            const float As = A_[(ys + k) * kCT + x];
            kword |= (__float_as_uint(As) == 0u ? 15u : (uint32_t)x_tier(As, B_[(ys + k) * kCT + x])) << (4 * k);
        }
        return tier_summary(kword);
    };
    bool failed = false;
    uint32_t ksum = 0u;       // this thread's tier summary at the current step
    float la[kM], lb[kM];     // scaled adjoint mu of this thread's cells (lambda = mu 2^sigma)
    uint32_t sgp[2];          // sigma at t + 1 of the 8 cells, 4 per word
    for (int l = 0; !failed; ++l) {
        // written by thread 0 before the barriers of the previous tile's steps
        const int ent = tring[l & 3];
        if (ent < 0) break;
        int r0, c0;
        origin(ent & kTileIndexMask, tiles_x, r0, c0);
        if (!__syncthreads_and(mbar_wait_bounded(&qbar, (uint32_t)(l & 1), hk.spin))) {
            failed = true;
            break;
        }
        // prologue: lambda' of the region -> registers (all loads issued before any
        // TMEM access, so they overlap), q -> TMEM, dL/dq accumulator := 0
        sgp[0] = sgp[1] = 0u;
#pragma unroll
        for (int k = 0; k < kM; ++k) {
            const int gr = r0 + ys + k, gc = c0 + x;
            const bool in = gr >= 0 && gr < H && gc >= 0 && gc < pitch;
            la[k] = in ? __ldg(lam_in + (size_t)gr * pitch + gc) : 0.0f;
            lb[k] = in ? __ldg(lam_in + gplane + (size_t)gr * pitch + gc) : 0.0f;
            const uint32_t sv = in ? (uint32_t)__ldg(sig_in + (size_t)gr * pitch + gc) : (uint32_t)kSigmaZero;
            sgp[k >> 2] |= sv << (8 * (k & 3));
        }
#pragma unroll
        for (int k = 0; k < kM; ++k) {
            const int y = ys + k;
            float qv[8], z[8];
#pragma unroll
            for (int d = 0; d < 8; ++d) {
                qv[d] = sm.q[d * kPlane + y * kCT + x];
                z[d] = 0.0f;
            }
            tmem_st8_nc(tbase + 16 * k, qv);
            tmem_st8_nc(tbase + 16 * k + 8, z);
        }
        // the tier summary of the tile's first step (the barrier below publishes it)
        bool pro_ok;
        {
            const int i0 = l * n;
            pro_ok = mbar_wait_bounded(&sbar[i0 & 1], (uint32_t)((i0 >> 1) & 1), hk.spin);
            ksum = tier_sum(sm.st[i0 & 1], sm.st[i0 & 1] + kPlane);
            sm.ks[i0 & 1][tid] = ksum;
        }
        tmem_wait_st();
        fence_proxy_async();
        if (!__syncthreads_and(pro_ok)) {  // q stage consumed; the first step's summaries
            failed = true;
            break;
        }
        if (tid == 0) issue_q(l + 1);

        for (int m = 0; m < n; ++m) {
            const int i = l * n + m;
            const int s = i & 1, ex = i & 1;
            // each thread waits for the stage itself; a wait that ran out is agreed on at
            // the step's barrier below (one barrier per step)
            const bool stage_ok = mbar_wait_bounded(&sbar[s], (uint32_t)((i >> 1) & 1), hk.spin);
            const float* stA = sm.st[s];
            const float* stB = sm.st[s] + kPlane;
            // every row but the region's edges is processed: skipping the rows the shrinking
            // halo no longer needs costs more in branching than it saves
            const int ylo = 1, yhi = kRT - 1;
            const bool xin = x >= 1 && x < kCT - 1;
            const int xl = xin ? x - 1 : x, xr = xin ? x + 1 : x;
            uint32_t sgc[2] = {0u, 0u};  // sigma at t of the 8 cells (from the staged state)
            float scl[kM];               // 2^(sigma(t+1) - sigma(t)) of each own cell (0 if masked)
            // contributions to source rows ys-1+R, as a ring of three rows (R = k, k+1,
            // k+2 while cell k is processed; slot R % 3) x three columns (x-1, x, x+1),
            // in the units of the source. Ring indices are compile-time constants.
            float w[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
            float own[kM];  // this thread's column, rows ys .. ys+7, before cross-warp / strip terms
            // b and 2^-sigma(t) of rows y-1, y, y+1 in columns x-1, x, x+1: ring slot (row - ys + 1) % 3
            // A warp whose windows (rows ys-1 .. ys+8, columns x-1 .. x+1) hold, at t, cells of
            // one tier k0 besides cells with a = 0, and whose cells are at t + 1 in tier k0 or
            // k0 - 1 (or have a = 0), needs no unit ratios between sources: every transfer of
            // a target j is rescaled by 2^(64 (sigma'(j) - k0)), folded into its l_P once.
            // Other warps take the general arithmetic, a ratio per transfer.
            uint32_t k0;
            bool uni = window_one_tier(sm.ks[s], tid, x - xl, xr - x, strip > 0, strip < kStrips - 1, kCT, ksum, k0);
            {
                // every byte of sigma' in {kSigmaZero, k0, k0 - 1}, four bytes a compare
                const uint32_t k4 = k0 * 0x01010101u, km4 = ((k0 - 1u) & 0xffu) * 0x01010101u;
#pragma unroll
                for (int w2 = 0; w2 < 2; ++w2) {
                    const uint32_t ok = __vcmpeq4(sgp[w2], 0xffffffffu) | __vcmpeq4(sgp[w2], k4) |
                                        __vcmpeq4(sgp[w2], km4);
                    uni = uni && ok == 0xffffffffu;
                }
            }
            const bool slow = !__all_sync(0xffffffffu, uni);
            auto cells = [&](auto tag) {
                constexpr bool kSlow = decltype(tag)::value;
                // stored b and (general path) the tier of rows y-1, y, y+1 in columns x-1, x,
                // x+1: ring slot (row - ys + 1) % 3
                float bw[3][3];
                int sw[3][3];
                auto src = [&](int row, int c, float& bv, int& sv) {
                    const int o = row * kCT + c;
                    bv = stB[o];
                    if constexpr (kSlow) sv = x_sigma(stA[o], bv);
                };
                {
                    const int y0 = ys > 0 ? ys - 1 : 0;
                    const int cols[3] = {xl, x, xr};
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        src(y0, cols[c], bw[0][c], sw[0][c]);
                        src(ys, cols[c], bw[1][c], sw[1][c]);
                    }
                }
#pragma unroll
                for (int k = 0; k < kM; ++k) {
                    const int y = ys + k;
                    float(&bu)[3] = bw[k % 3];
                    float(&bm)[3] = bw[(k + 1) % 3];
                    float(&bd)[3] = bw[(k + 2) % 3];
                    int(&su)[3] = sw[k % 3];
                    int(&sm3)[3] = sw[(k + 1) % 3];
                    int(&sd)[3] = sw[(k + 2) % 3];
                    {
                        const int yd = y + 1 < kRT ? y + 1 : y;
                        const int cols[3] = {xl, x, xr};
#pragma unroll
                        for (int c = 0; c < 3; ++c) src(yd, cols[c], bd[c], sd[c]);
                    }
                    float(&wu)[3] = w[k % 3];        // source row y - 1 (R = k)
                    float(&wm)[3] = w[(k + 1) % 3];  // source row y
                    float(&wd)[3] = w[(k + 2) % 3];  // source row y + 1
                    const float Aown = stA[y * kCT + x];
                    // sigma(t) of this cell: the tier (k0 on the single-tier path), kSigmaZero for a = 0
                    int sg;
                    if constexpr (kSlow) sg = sm3[1];
                    else sg = __float_as_uint(Aown) == 0u ? kSigmaZero : (int)k0;
                    sgc[k >> 2] |= (uint32_t)sg << (8 * (k & 3));
                    const int sp = (int)((sgp[k >> 2] >> (8 * (k & 3))) & 0xffu);
                    const bool live = sp != kSigmaZero;  // a > 0 at t + 1
                    // single tier: 2^(64 (sigma'(j) - k0)), the ratio of every transfer of j and,
                    // for this cell's own l_a, the ratio 2^(64 (sigma'(j) - sigma(j)))
                    const float Up = (kSlow || !live) ? 0.0f : (sp == (int)k0 ? 1.0f : 0x1p-64f);
                    scl[k] = (sg == kSigmaZero || !live) ? 0.0f : (kSlow ? exp2i(64 * (sp - sg)) : Up);
                    uint32_t tmv[16];
                    tmem_ld16_async(tbase + 16 * k, tmv);
                    tmem_wait_ld16(tmv);
                    if (y >= ylo && y < yhi) {  // uniform across the warp
                        float qv[8], gv[8];
#pragma unroll
                        for (int d = 0; d < 8; ++d) {
                            qv[d] = __uint_as_float(tmv[d]);
                            gv[d] = __uint_as_float(tmv[8 + d]);
                        }
                        // neighbours in direction order (-1,-1) (-1,0) (-1,1) (0,-1) (0,1) (1,-1) (1,0) (1,1)
                        const float nb[8] = {bu[0], bu[1], bu[2], bm[0], bm[2], bd[0], bd[1], bd[2]};
                        // no neighbour with b in tier 0 (b = 0, or a tiered b below 2^-64,
                        // stored negative): every factor 1 - b_i q_dj is exactly 1. The short
                        // path below is taken when that holds for every cell of the warp's row
                        // that has a > 0 at t + 1; otherwise the whole row takes the general
                        // arithmetic, which gives the short path's bits on such cells (so a row
                        // of both kinds does not run both paths one after the other).
                        float nbmax = nb[0];
#pragma unroll
                        for (int d = 1; d < 8; ++d) nbmax = fmaxf(nbmax, nb[d]);
                        const bool quiet = __all_sync(0xffffffffu, nbmax <= 0.0f || !live);
                        if (live) {
                            // The region's edge columns (!xin) contribute nothing: they take
                            // the same path on their clamped (in-bounds) window with tg = 0 and
                            // P = 0, which leaves only l_a <- l_a scl, instead of diverging.
                            float r[8];  // 2^(64 (sigma'(j) - sigma(i))): to the units of source i
                            if constexpr (kSlow) {
                                const int ns[8] = {su[0], su[1], su[2], sm3[0], sm3[2], sd[0], sd[1], sd[2]};
#pragma unroll
                                for (int d = 0; d < 8; ++d) r[d] = exp2i(64 * (sp - ns[d]));
                            }
                            // 1 - a of this cell (1 in the tiers below 2^-64)
                            const bool own_tiered = kSlow ? (int32_t)__float_as_uint(bm[1]) < 0 : k0 != 0u;
                            const float ua = signbit(Aown) ? -Aown : (own_tiered ? 1.0f : 1.0f - Aown);
                            const float ln = la[k] + lb[k];
                            // l_P_j in units 2^(64 sigma'(j)); on the single-tier path already in
                            // the sources' units
                            const float tg = xin ? (kSlow ? ln * ua : (ln * ua) * Up) : 0.0f;
                            if (quiet) {
                                // P = 0 and every leave-one-out product is exactly 1, so t_d = tg:
                                // the general arithmetic below with its factors folded (the same
                                // bits); the dL/dq terms carry the tiered b_i (0 for b_i = 0)
                                la[k] *= scl[k];
                                {  // tg = 0 (edge columns; cells burned out to a = 1 exactly) adds zeros
#pragma unroll
                                    for (int d = 0; d < 8; ++d) {
                                        const float g = kSlow ? fabsf(nb[d]) * r[d] : fabsf(nb[d]);
                                        gv[d] = fmaf(tg, g, gv[d]);
                                        const float tqv = tg * qv[d];
                                        const float c = kSlow ? tqv * r[d] : tqv;
                                        const int j = dir_dc(d) + 1;
                                        if (dir_dr(d) < 0) wu[j] += c;
                                        else if (dir_dr(d) == 0) wm[j] += c;
                                        else wd[j] += c;
                                    }
                                }
                            } else {
                                float f[8];
                                // b of a tiered source is below 2^-64: its factor is exactly 1
#pragma unroll
                                for (int d = 0; d < 8; ++d) f[d] = fmaf(-fmaxf(nb[d], 0.0f), qv[d], 1.0f);
                                // t_d = tg prod_{e != d} f_e by a product tree over pairs and
                                // halves (no division: a factor can be exactly 0)
                                const float p01 = f[0] * f[1], p23 = f[2] * f[3], p45 = f[4] * f[5], p67 = f[6] * f[7];
                                const float p03 = p01 * p23, p47 = p45 * p67;
                                // P enters only l_a = l_a' - l_n P here, where 1 - S's absolute
                                // error (a few 1e-8) is harmless; the forward keeps the recurrence
                                const float P = xin ? 1.0f - p03 * p47 : 0.0f;
                                la[k] = fmaf(-ln, P, la[k]) * scl[k];
                                {  // as above: unconditional, tg = 0 adds zeros
                                    const float g03 = tg * p47, g47 = tg * p03;
                                    const float r01 = g03 * p23, r23 = g03 * p01, r45 = g47 * p67, r67 = g47 * p45;
                                    const float t[8] = {f[1] * r01, f[0] * r01, f[3] * r23, f[2] * r23,
                                                        f[5] * r45, f[4] * r45, f[7] * r67, f[6] * r67};
#pragma unroll
                                    for (int d = 0; d < 8; ++d) {
                                        // dL/dq_dj += l_P_j b_i prod_{e != d} f_e, b_i = |B_i| 2^(-64 sigma(i))
                                        const float g = kSlow ? fabsf(nb[d]) * r[d] : fabsf(nb[d]);
                                        gv[d] = fmaf(t[d], g, gv[d]);
                                        const float tqv = t[d] * qv[d];
                                        const float c = kSlow ? tqv * r[d] : tqv;
                                        const int j = dir_dc(d) + 1;
                                        if (dir_dr(d) < 0) wu[j] += c;
                                        else if (dir_dr(d) == 0) wm[j] += c;
                                        else wd[j] += c;
                                    }
                                }
                            }
                        } else {
                            la[k] *= scl[k];
                        }
                        tmem_st8_nc(tbase + 16 * k + 8, gv);
                    } else {
                        la[k] *= scl[k];
                    }
                    // row R = k (source row ys + k - 1) is complete
                    if (k == 0) {
#pragma unroll
                        for (int j = 0; j < 3; ++j) sm.vtop[ex][strip][j][x] = wu[j];
                    } else {
                        const float fr = __shfl_down_sync(0xffffffffu, wu[0], 1);  // from column x + 1
                        const float fl = __shfl_up_sync(0xffffffffu, wu[2], 1);    // from column x - 1
                        own[k - 1] = wu[1] + (lane < 31 ? fr : 0.0f) + (lane > 0 ? fl : 0.0f);
                        exchange(ex, k - 1, wu[2], wu[0]);
                    }
#pragma unroll
                    for (int j = 0; j < 3; ++j) wu[j] = 0.0f;  // the slot becomes row R = k + 3
                }
            };
            if (slow) cells(std::true_type{});
            else cells(std::false_type{});
            // rows R = 8 (source row ys + 7, slot 8 % 3) and R = 9 (the next strip's first row)
            {
                float(&w8)[3] = w[kM % 3];
                float(&w9)[3] = w[(kM + 1) % 3];
                const float fr = __shfl_down_sync(0xffffffffu, w8[0], 1);
                const float fl = __shfl_up_sync(0xffffffffu, w8[2], 1);
                own[kM - 1] = w8[1] + (lane < 31 ? fr : 0.0f) + (lane > 0 ? fl : 0.0f);
                exchange(ex, kM - 1, w8[2], w8[0]);
#pragma unroll
                for (int j = 0; j < 3; ++j) sm.vbot[ex][strip][j][x] = w9[j];
            }
            // the next step's tier summary, published by this step's end barrier
            bool next_ok = true;
            if (m + 1 < n) {
                const int s1 = (i + 1) & 1;
                next_ok = mbar_wait_bounded(&sbar[s1], (uint32_t)(((i + 1) >> 1) & 1), hk.spin);
                ksum = tier_sum(sm.st[s1], sm.st[s1] + kPlane);
                sm.ks[s1][tid] = ksum;
            }
            tmem_wait_st();
            fence_proxy_async();  // stage s fully read before it is refilled by TMA
            if (!__syncthreads_and(stage_ok && next_ok)) {
                failed = true;
                break;
            }
            if (tid == 0) issue_state(i + 2);
            // gather: lambda_b at the sources of this strip. The per-lane boundary terms are
            // selected rather than branched on: every lane loads them (one address per warp,
            // a broadcast) and keeps its own.
            const int xp = x + 1 < kCT ? x + 1 : x, xm = x >= 1 ? x - 1 : x;
            // bytes of sigma(t) equal to kSigmaZero (a = 0), as 0xff masks
            const uint32_t dmask[2] = {__vcmpeq4(sgc[0], 0xffffffffu), __vcmpeq4(sgc[1], 0xffffffffu)};
            // the cross-warp terms of this strip's 8 rows: x = 31 takes those from x = 32, x =
            // 32 those from x = 31, the others add zeros (two 16-byte loads a thread)
            const bool edge = x == 31 || x == 32;
            const float4* ep = reinterpret_cast<const float4*>(x == 31 ? sm.er2l[ex][strip] : sm.el2r[ex][strip]);
            const float4 e0 = ep[0], e1 = ep[1];
            const float ev[kM] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
#pragma unroll
            for (int k = 0; k < kM; ++k) {
                float v = fmaf(pc * scl[k], lb[k], own[k]);
                v += edge ? ev[k] : 0.0f;
                if (k == 0 && strip > 0) {  // uniform across the warp
                    const float c = sm.vbot[ex][strip - 1][1][x];
                    const float r = sm.vbot[ex][strip - 1][0][xp], lf = sm.vbot[ex][strip - 1][2][xm];
                    v += c;
                    v += x + 1 < kCT ? r : 0.0f;
                    v += x >= 1 ? lf : 0.0f;
                }
                if (k == kM - 1 && strip < kStrips - 1) {
                    const float c = sm.vtop[ex][strip + 1][1][x];
                    const float r = sm.vtop[ex][strip + 1][0][xp], lf = sm.vtop[ex][strip + 1][2][xm];
                    v += c;
                    v += x + 1 < kCT ? r : 0.0f;
                    v += x >= 1 ? lf : 0.0f;
                }
                // a == 0 at t: lambda multiplies only zeros
                const bool dead = (dmask[k >> 2] >> (8 * (k & 3))) & 1u;
                lb[k] = dead ? 0.0f : v;
                la[k] = dead ? 0.0f : la[k];
            }
            sgp[0] = sgc[0];
            sgp[1] = sgc[1];
        }
        if (failed) break;
        // lambda at t0 and the tile's dL/dq for the interior
        const bool xint = x >= kHalo && x < kCT - kHalo;
#pragma unroll
        for (int k = 0; k < kM; ++k) {
            const int y = ys + k;
            float gv[8];
            tmem_ld8(tbase + 16 * k + 8, gv);
            const int gr = r0 + y, gc = c0 + x;
            if (xint && y >= kHalo && y < kRT - kHalo && gr < H && gc < pitch) {
                const size_t j = (size_t)gr * pitch + gc;
                lam_out[j] = la[k];
                lam_out[gplane + j] = lb[k];
                sig_out[j] = (uint8_t)((sgp[k >> 2] >> (8 * (k & 3))) & 0xffu);
                // fire-and-forget reductions (no load round trip); each cell receives
                // exactly one add per launch, so the result does not depend on timing
#pragma unroll
                for (int d = 0; d < 8; ++d) atomicAdd(Gq + d * gplane + j, gv[d]);
            }
        }
    }
    if (failed && tid == 0) {
        atomicExch(err, kErrTmaTimeout);
        // give the copies in flight one more bounded wait before the CTA exits
        mbar_wait_bounded(&qbar, 0, hk.spin);
        mbar_wait_bounded(&sbar[0], 0, hk.spin);
        mbar_wait_bounded(&sbar[1], 0, hk.spin);
    }
    tmem_sync_threads();
    if (warp == 0) tmem_dealloc(tslot, kTmemCols);
}

// ---------------------------------------------------------------- frozen tiles
// The tiles the pre-pass lists from the back of the tile list (kTileFrozenBit): the
// region's state is constant over the launch and b = 0 in it, so sigma(t) = sigma(t + 1),
// P = 0, every leave-one-out product is 1 and no dL/dq term survives. A step reduces to
//   l_b,i <- p_c l_b,i + sum_d G_di (l_a + l_b)_(i - dir d),   l_a unchanged,
// over the sources i, with the targets j = i - dir(d) and the constant coefficients
// G_di = (1 - a_j) q_dj 2^(64 (sigma_j - sigma_i)) (0 for targets on the region's edge,
// with a = 0, or outside the grid). This kernel runs them apart from the live tiles: no
// tensor memory and no cross-lane exchange. The region's q, state and lambda are staged
// by TMA during the previous tile's steps; G stays in registers and l_a + l_b goes
// through two zero-bordered shared-memory planes (a step reads one and writes the other,
// one barrier a step).
constexpr int kFM = 8;                              // rows per thread
constexpr int kFThreads = kCT * (kRT / kFM);        // 512
struct FrozenSmem {
    float q[8 * kPlane];            // q stage (TMA)
    float st[2 * kPlane];           // state stage (TMA); then 1 - a and sigma (as int bits) in place
    float lam[2 * kPlane];          // lambda stage (TMA)
    float ln[2][kRT + 2][kCT + 2];  // l_a + l_b of the region, by step parity; the borders stay 0
};
static_assert(sizeof(FrozenSmem) + 128 <= 227 * 1024, "k_adjoint_frozen's shared memory");

__global__ void __launch_bounds__(kFThreads, 1)
    k_adjoint_frozen(const __grid_constant__ CUtensorMap tst, const __grid_constant__ CUtensorMap tst0,
                     const __grid_constant__ CUtensorMap tq, const __grid_constant__ CUtensorMap tlam, int H,
                     int pitch, float pc, int zlast, int n, int tiles_x, const int* __restrict__ tiles,
                     const int* __restrict__ counts, int* __restrict__ work, float* __restrict__ lam_out,
                     uint8_t* __restrict__ sig_out, int* __restrict__ err, TmaHook hk) {
    extern __shared__ __align__(128) uint8_t fraw[];
    FrozenSmem& sm = *reinterpret_cast<FrozenSmem*>(fraw + ((128u - (smem_u32(fraw) & 127u)) & 127u));
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_next;
    // least and greatest sigma of the region's cells with a > 0 (reset for every tile)
    __shared__ unsigned s_tlo, s_thi;
    const int nfz = counts[2];
    int k = blockIdx.x;
    if (k >= nfz) return;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int x = tid % kCT;
    const int ys = (tid / kCT) * kFM;
    const size_t plane = (size_t)H * pitch;
    const int cap = tiles_x * ((H + kIR - 1) / kIR);  // the list's capacity
    const uint32_t bytes = (uint32_t)((8 + 2 + 2) * kPlane * sizeof(float));
    // thread 0: stage tile list entry k (q, the launch's first state, lambda at t + 1)
    auto issue = [&](int kk) {
        const int e = tiles[cap - 1 - kk];
        int r0, c0;
        origin(e & kTileIndexMask, tiles_x, r0, c0);
        // the launch's first state; state 0 when the region has not changed since then
        const int z = (e & kTileCkptBit) ? 0 : zlast - (n - 1);
        mbar_arrive_expect_tx(&bar, bytes);
        if (hk.withhold) return;
        tma_load_3d(sm.q, &tq, &bar, c0, r0, 0);
        if (z == 0) tma_load_3d(sm.st, &tst0, &bar, c0, r0, 0);
        else tma_load_3d(sm.st, &tst, &bar, c0, r0, 2 * z);
        tma_load_3d(sm.lam, &tlam, &bar, c0, r0, 0);
    };
    for (int i = tid; i < 2 * (kRT + 2) * (kCT + 2); i += kFThreads) (&sm.ln[0][0][0])[i] = 0.0f;
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        issue(k);
        s_next = (int)gridDim.x + atomicAdd(work, 1);
        s_tlo = 255u;
        s_thi = 0u;
    }
    __syncthreads();
    uint32_t parity = 0u;
    float* stA = sm.st;
    float* stB = sm.st + kPlane;
    while (k < nfz) {
        const int next = s_next;  // written before the previous barrier
        int r0, c0;
        origin(tiles[cap - 1 - k] & kTileIndexMask, tiles_x, r0, c0);
        if (!__syncthreads_and(mbar_wait_bounded(&bar, parity, hk.spin))) {
            if (tid == 0) {
                atomicExch(err, kErrTmaTimeout);
                mbar_wait_bounded(&bar, parity, hk.spin);  // the copies in flight get one more budget
            }
            return;
        }
        parity ^= 1u;
        // stage -> registers and planes: lambda (0 where a = 0), 1 - a (0 where a = 0) and
        // sigma in place
        float la[kFM], lb[kFM];
        uint32_t sgp[kFM / 4] = {};  // sigma of the cells (at t and t + 1 alike), a byte each
        unsigned tlo = 255u, thi = 0u;
#pragma unroll
        for (int m = 0; m < kFM; ++m) {
            const int o = (ys + m) * kCT + x;
            const float A = stA[o], B = stB[o];
            const int sg = x_sigma(A, B);
            const bool lv = sg != kSigmaZero;
            la[m] = lv ? sm.lam[o] : 0.0f;
            lb[m] = lv ? sm.lam[kPlane + o] : 0.0f;
            sgp[m >> 2] |= (uint32_t)sg << (8 * (m & 3));
            sm.ln[0][ys + m + 1][x + 1] = la[m] + lb[m];
            stA[o] = !lv ? 0.0f : (signbit(A) ? -A : ((int32_t)__float_as_uint(B) < 0 ? 1.0f : 1.0f - A));
            stB[o] = __int_as_float(sg);
            tlo = min(tlo, (unsigned)sg);            // kSigmaZero is the greatest value
            thi = max(thi, lv ? (unsigned)sg : 0u);
        }
        tlo = __reduce_min_sync(0xffffffffu, tlo);
        thi = __reduce_max_sync(0xffffffffu, thi);
        if (lane == 0) {
            atomicMin(&s_tlo, tlo);
            atomicMax(&s_thi, thi);
        }
        __syncthreads();
        // one sigma for every cell with a > 0 in the region (or none): every transfer's
        // unit ratio is 1 and a target with a = 0 has 1 - a stored as 0, so G needs no sigma
        const bool one_tier = s_tlo >= s_thi;
        // the coefficients of this thread's sources
        float G[kFM][8];
        if (one_tier) {
#pragma unroll
            for (int m = 0; m < kFM; ++m) {
                const int y = ys + m;
                const bool si_live = ((sgp[m >> 2] >> (8 * (m & 3))) & 0xffu) != (uint32_t)kSigmaZero;
#pragma unroll
                for (int d = 0; d < 8; ++d) {
                    const int jy = y - dir_dr(d), jx = x - dir_dc(d);
                    const bool inr = jy >= 1 && jy < kRT - 1 && jx >= 1 && jx < kCT - 1;
                    const int oj = inr ? jy * kCT + jx : 0;
                    G[m][d] = (si_live && inr) ? stA[oj] * sm.q[d * kPlane + oj] : 0.0f;
                }
            }
        } else {
#pragma unroll
            for (int m = 0; m < kFM; ++m) {
                const int y = ys + m;
                const int si = (int)((sgp[m >> 2] >> (8 * (m & 3))) & 0xffu);
#pragma unroll
                for (int d = 0; d < 8; ++d) {
                    const int jy = y - dir_dr(d), jx = x - dir_dc(d);
                    // targets on the region's edge rows and columns contribute nothing
                    const bool inr = jy >= 1 && jy < kRT - 1 && jx >= 1 && jx < kCT - 1;
                    const int oj = inr ? jy * kCT + jx : 0;
                    const int sj = inr ? __float_as_int(stB[oj]) : kSigmaZero;
                    const bool use = si != kSigmaZero && sj != kSigmaZero;
                    G[m][d] = use ? (stA[oj] * sm.q[d * kPlane + oj]) * exp2i(64 * (sj - si)) : 0.0f;
                }
            }
        }
        fence_proxy_async();  // these generic reads of the stages precede the next TMA writes
        __syncthreads();      // every stage fully read
        if (tid == 0 && next < nfz) issue(next);
        // the steps: rows ys-1 .. ys+kFM of l_a + l_b in columns x-1, x, x+1 read from one
        // plane, the new values written into the other
        for (int s = 0; s < n; ++s) {
            const int p = s & 1;
            float w[kFM + 2][3];
            // the thread's own column (rows ys .. ys+7) is what it wrote last: la + lb
#pragma unroll
            for (int r = 0; r < kFM + 2; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    w[r][c] = (c == 1 && r >= 1 && r <= kFM) ? la[r - 1] + lb[r - 1] : sm.ln[p][ys + r][x + c];
#pragma unroll
            for (int m = 0; m < kFM; ++m) {
                // target i - dir(d) of source (ys + m, x) sits at window (m + 1 - dr, 1 - dc)
                float own = 0.0f;
#pragma unroll
                for (int d = 0; d < 8; ++d) own = fmaf(G[m][d], w[m + 1 - dir_dr(d)][1 - dir_dc(d)], own);
                const bool lv = ((sgp[m >> 2] >> (8 * (m & 3))) & 0xffu) != (uint32_t)kSigmaZero;
                lb[m] = lv ? fmaf(pc, lb[m], own) : 0.0f;
                sm.ln[p ^ 1][ys + m + 1][x + 1] = la[m] + lb[m];
            }
            __syncthreads();  // the new plane complete, the old one read by every thread
        }
        // lambda at t0 of the interior (sigma unchanged); a frozen tile adds no dL/dq
        const int gc = c0 + x;
        if (x >= kHalo && x < kCT - kHalo && gc < pitch) {
#pragma unroll
            for (int m = 0; m < kFM; ++m) {
                const int y = ys + m, gr = r0 + y;
                if (y >= kHalo && y < kRT - kHalo && gr < H) {
                    const size_t j = (size_t)gr * pitch + gc;
                    lam_out[j] = la[m];
                    lam_out[plane + j] = lb[m];
                    sig_out[j] = (uint8_t)((sgp[m >> 2] >> (8 * (m & 3))) & 0xffu);
                }
            }
        }
        if (tid == 0) {
            if (next < nfz) s_next = (int)gridDim.x + atomicAdd(work, 1);
            s_tlo = 255u;
            s_thi = 0u;
        }
        __syncthreads();  // s_next, the sigma bounds reset
        k = next;
    }
}

// Pre-pass of one adjoint launch: for each tile, whether any cell of its 64 x 64 region
// has a > 0 in the latest state of the launch's steps (A at t1 - 1, the encoded a plane).
// a never decreases in time, so a tile with a = 0 in its whole region has a = b = 0 there
// at every step of the launch: all its lambdas end masked to 0 and every dL/dq term
// carries a factor b_i = 0. Such a tile's interior gets lambda = 0, sigma = kSigmaZero
// here; the others are listed (in any order: each tile writes only its own interior and
// adds to its own cells' dL/dq once) for k_adjoint_blocked.
__device__ __forceinline__ void adjoint_tile(const float* __restrict__ A, int H, int W, int pitch,
                                                       int tiles_x, int ntiles, int n, int* __restrict__ list,
                                                       int* __restrict__ count, float* __restrict__ lam_out,
                                                       uint8_t* __restrict__ sig_out, uint8_t* __restrict__ gq_dirty,
                                                       unsigned long long* __restrict__ skipped, int tile, int lane,
                                                       unsigned long long& sk) {
    int r0, c0;
    origin(tile, tiles_x, r0, c0);
    uint32_t any = 0u;
    // 64 rows x 16 float4 (c0 and pitch are multiples of 4 floats: a float4 is wholly
    // inside or wholly outside [0, pitch))
    for (int i = lane; i < kRT * (kCT / 4); i += 32) {
        const int gr = r0 + i / (kCT / 4), gc = c0 + 4 * (i % (kCT / 4));
        if (gr < 0 || gr >= H || gc < 0 || gc >= pitch) continue;
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(A + (size_t)gr * pitch + gc));
        any |= v.x | v.y | v.z | v.w;
    }
    if (__any_sync(0xffffffffu, any != 0u)) {
        if (lane == 0) {
            list[atomicAdd(count, 1)] = tile;
            if (gq_dirty) gq_dirty[tile] = 1;
        }
        return;
    }
    const size_t gplane = (size_t)H * pitch;
    const int ir0 = r0 + kHalo, ic0 = c0 + kHalo;
    for (int i = lane; i < kIR * (kIC / 4); i += 32) {
        const int gr = ir0 + i / (kIC / 4), gc = ic0 + 4 * (i % (kIC / 4));
        if (gr >= H || gc >= pitch) continue;
        const size_t j = (size_t)gr * pitch + gc;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        *reinterpret_cast<float4*>(lam_out + j) = z;
        *reinterpret_cast<float4*>(lam_out + gplane + j) = z;
        *reinterpret_cast<uint32_t*>(sig_out + j) = 0x01010101u * (uint32_t)kSigmaZero;
    }
    if (lane == 0) sk = (unsigned long long)(min(kIR, H - ir0) * min(kIC, W - ic0)) * (unsigned long long)n;
}

__global__ void __launch_bounds__(256) k_adjoint_tiles(const float* __restrict__ A, int H, int W, int pitch,
                                                       int tiles_x, int ntiles, int n, int* __restrict__ list,
                                                       int* __restrict__ count, float* __restrict__ lam_out,
                                                       uint8_t* __restrict__ sig_out, uint8_t* __restrict__ gq_dirty,
                                                       unsigned long long* __restrict__ skipped) {
    __shared__ unsigned long long s_sk;
    if (threadIdx.x == 0) s_sk = 0ull;
    __syncthreads();
    unsigned long long sk = 0ull;
    const int tile = blockIdx.x * 8 + (threadIdx.x >> 5);  // one warp per tile
    if (tile < ntiles)
        adjoint_tile(A, H, W, pitch, tiles_x, ntiles, n, list, count, lam_out, sig_out, gq_dirty, skipped, tile,
                     threadIdx.x & 31, sk);
    block_count(skipped, s_sk, sk);
}

__device__ __forceinline__ void adjoint_tile_flags(const uint8_t* __restrict__ act, int H, int W, int pitch,
                                                             int tiles_x, int tiles_y, int n, int* __restrict__ list,
                                                             int* __restrict__ count, float* __restrict__ lam_out,
                                                             uint8_t* __restrict__ sig_out,
                                                             uint8_t* __restrict__ deadcnt, int use_frozen,
                                                             uint8_t* __restrict__ gq_dirty,
                                                             unsigned long long* __restrict__ skipped,
                                                             unsigned long long* __restrict__ frozen_steps, int tile,
                                                             int lane, unsigned long long& sk,
                                                             unsigned long long& fz_steps) {
    const int ty = tile / tiles_x, tx = tile % tiles_x;
    // the tile's quiescent count, loaded with the flags below so that the latencies overlap
    const int dc = deadcnt[tile];
    // the 3 x 3 flags around the tile, one per lane: OR-reduced, and whether all of them
    // are unchanged since the segment's first state (kQb; outside the grid: yes)
    uint32_t f = 0u, qb = 1u;
    if (lane < 9) {
        const int yy = ty + lane / 3 - 1, xx = tx + lane % 3 - 1;
        if (yy >= 0 && yy < tiles_y && xx >= 0 && xx < tiles_x) {
            f = act[yy * tiles_x + xx];
            qb = (f & kQb) ? 1u : 0u;
        }
    }
    const uint32_t me = __shfl_sync(0xffffffffu, f, 4);  // lane 4 holds the tile's own flags
    const uint32_t around = __reduce_or_sync(0xffffffffu, f);
    const bool all_qb = __reduce_and_sync(0xffffffffu, qb) != 0u;
    if (around & kActA) {
        if (lane == 0) {
            const bool fz = use_frozen && (me & kFrozen);
            const int cap = tiles_x * tiles_y;  // the list's capacity
            if (fz)  // from the back of the list (count[2] of them)
                list[cap - 1 - atomicAdd(count + 2, 1)] = tile | kTileFrozenBit | (all_qb ? kTileCkptBit : 0);
            else
                list[atomicAdd(count, 1)] = tile;
            deadcnt[tile] = 0;
            if (gq_dirty && !fz) gq_dirty[tile] = 1;
            if (fz) {
                int r0, c0;
                origin(tile, tiles_x, r0, c0);
                fz_steps = (unsigned long long)(min(kIR, H - r0 - kHalo) * min(kIC, W - c0 - kHalo)) *
                           (unsigned long long)n;
            }
        }
        return;
    }
    int r0, c0;
    origin(tile, tiles_x, r0, c0);
    const int ir0 = r0 + kHalo, ic0 = c0 + kHalo;
    if (dc < 2) {  // the first two quiescent launches fill both ping-pong buffers
        const size_t gplane = (size_t)H * pitch;
        for (int i = lane; i < kIR * (kIC / 4); i += 32) {
            const int gr = ir0 + i / (kIC / 4), gc = ic0 + 4 * (i % (kIC / 4));
            if (gr >= H || gc >= pitch) continue;
            const size_t j = (size_t)gr * pitch + gc;
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<float4*>(lam_out + j) = z;
            *reinterpret_cast<float4*>(lam_out + gplane + j) = z;
            *reinterpret_cast<uint32_t*>(sig_out + j) = 0x01010101u * (uint32_t)kSigmaZero;
        }
    }
    __syncwarp();
    if (lane == 0) {
        if (dc < 2) deadcnt[tile] = (uint8_t)(dc + 1);
        sk = (unsigned long long)(min(kIR, H - ir0) * min(kIC, W - ic0)) * (unsigned long long)n;
    }
}

__global__ void __launch_bounds__(256) k_adjoint_tiles_flags(const uint8_t* __restrict__ act, int H, int W, int pitch,
                                                             int tiles_x, int tiles_y, int n, int* __restrict__ list,
                                                             int* __restrict__ count, float* __restrict__ lam_out,
                                                             uint8_t* __restrict__ sig_out,
                                                             uint8_t* __restrict__ deadcnt, int use_frozen,
                                                             uint8_t* __restrict__ gq_dirty,
                                                             unsigned long long* __restrict__ skipped,
                                                             unsigned long long* __restrict__ frozen_steps) {
    __shared__ unsigned long long s_sk, s_fz;
    if (threadIdx.x == 0) s_sk = s_fz = 0ull;
    __syncthreads();
    unsigned long long sk = 0ull, fz = 0ull;
    const int tile = blockIdx.x * 8 + (threadIdx.x >> 5);  // one warp per tile
    if (tile < tiles_x * tiles_y)
        adjoint_tile_flags(act, H, W, pitch, tiles_x, tiles_y, n, list, count, lam_out, sig_out, deadcnt, use_frozen,
                           gq_dirty, skipped, frozen_steps, tile, threadIdx.x & 31, sk, fz);
    block_count(skipped, s_sk, sk);
    block_count(frozen_steps, s_fz, fz);
}

}  // namespace

int adjoint_blocked_max_steps() { return kMaxSteps; }

static size_t adjoint_blocked_smem() { return sizeof(Smem) + 128; }

int adjoint_blocked_configure() {
    static int done = 0;
    if (!done) {
        if (cudaFuncSetAttribute(k_adjoint_blocked, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)adjoint_blocked_smem()) != cudaSuccess ||
            cudaFuncSetAttribute(k_adjoint_frozen, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(FrozenSmem) + 128) != cudaSuccess)
            return -1;
        done = 1;
    }
    return 0;
}

int adjoint_blocked_tiles(int H, int pitch) { return ((pitch + kIC - 1) / kIC) * ((H + kIR - 1) / kIR); }

void launch_adjoint_tiles(const float* A_latest, int H, int W, int pitch, int n, float* lam_out, uint8_t* sig_out,
                          int* tile_list, int* tile_count, uint8_t* gq_dirty, unsigned long long* skipped,
                          cudaStream_t s) {
    const int tiles_x = (pitch + kIC - 1) / kIC;
    // the counts and both adjoint kernels' work counters
    cudaMemsetAsync(tile_count, 0, 4 * sizeof(int), s);
    const int ntiles = adjoint_blocked_tiles(H, pitch);
    k_adjoint_tiles<<<(ntiles + 7) / 8, 256, 0, s>>>(A_latest, H, W, pitch, tiles_x, ntiles, n, tile_list, tile_count,
                                                     lam_out, sig_out, gq_dirty, skipped);
}

void launch_adjoint_tiles_flags(const uint8_t* act, int H, int W, int pitch, int n, float* lam_out, uint8_t* sig_out,
                                uint8_t* deadcnt, int* tile_list, int* tile_count, bool use_frozen,
                                uint8_t* gq_dirty, unsigned long long* skipped, unsigned long long* frozen_steps,
                                cudaStream_t s) {
    const int tiles_x = (pitch + kIC - 1) / kIC, tiles_y = (H + kIR - 1) / kIR;
    const int ntiles = tiles_x * tiles_y;
    cudaMemsetAsync(tile_count, 0, 4 * sizeof(int), s);  // the counts and both adjoint kernels' work counters
    k_adjoint_tiles_flags<<<(ntiles + 7) / 8, 256, 0, s>>>(act, H, W, pitch, tiles_x, tiles_y, n, tile_list, tile_count,
                                                           lam_out, sig_out, deadcnt, use_frozen ? 1 : 0, gq_dirty,
                                                           skipped, frozen_steps);
}

void launch_adjoint_blocked(const CUtensorMap* tst, const CUtensorMap* tst0, const CUtensorMap* tq,
                            const CUtensorMap* tlam, int H, int pitch, float pc, int zlast, int n,
                            const float* lam_in, const uint8_t* sig_in, float* lam_out, uint8_t* sig_out, float* Gq,
                            const int* tile_list, int* tile_count, int nsm, int* err, TmaHook hk, bool frozen_only,
                            cudaStream_t s) {
    const int tiles_x = (pitch + kIC - 1) / kIC;
    const int ntiles = adjoint_blocked_tiles(H, pitch);
    const int grid = ntiles < nsm ? ntiles : nsm;
    if (!frozen_only)
        k_adjoint_blocked<<<grid, kThreads, adjoint_blocked_smem(), s>>>(*tst, *tst0, *tq, H, pitch, pc, zlast, n,
                                                                         tiles_x, tile_list, tile_count,
                                                                         tile_count + 1, lam_in, sig_in, lam_out,
                                                                         sig_out, Gq, err, hk);
    else
        k_adjoint_frozen<<<grid, kFThreads, sizeof(FrozenSmem) + 128, s>>>(*tst, *tst0, *tq, *tlam, H, pitch, pc,
                                                                           zlast, n, tiles_x, tile_list, tile_count,
                                                                           tile_count + 3, lam_out, sig_out, err, hk);
}

}  // namespace pf
