// Temporal-blocked differentiable forward step (the same update as k_diff_step, k
// steps per launch).
//
// Persistent kernel, one CTA per SM. Each CTA walks a static list of 48 x 48-cell
// interior tiles; for each it stages the 64 x 64 region (8-cell halo) of the state
// (A, b) and of the eight q planes in shared memory with two TMA tile loads, prefetching
// the next tile while it computes the current one. Each of the 512 threads owns an
// 8-cell column strip of the region and keeps its cells' q (64 floats) and encoded a
// in registers for the whole launch; b is exchanged through a shared-memory
// ping-pong buffer, read through a rolling 3 x 3 register window (3 shared loads per
// cell and step). After n <= 8 steps the interior, which is exact by then, is stored.
// Cells outside the grid arrive as TMA zero fill (q = 0, a = b = 0) and stay 0.
#include <cuda.h>

#include "common.cuh"
#include "prep_math.cuh"
#include "tma.cuh"

namespace pf {

namespace {

constexpr int kRT = 64, kCT = 64;      // staged region
// halo rows / columns = max steps per launch: 8 (interior 48 x 48) or, for launches of
// at most 4 steps, 4 (interior 56 x 56: 1.31x instead of 1.78x redundant halo work).
// Both keep the tile origins' columns multiples of 4 floats (16 B), as TMA requires.
constexpr int kHaloMax = 8;
constexpr int kM = 8;                  // cells per thread (column strip)
constexpr int kThreads = kCT * (kRT / kM);  // 512
constexpr int kPlane = kRT * kCT;      // floats per staged plane

struct Smem {
    float q[8 * kPlane];     // staged q planes of the next tile (TMA destination)
    float st[2 * kPlane];    // staged (A, b) of the next tile (TMA destination)
    float b[2][kPlane];      // b ping-pong of the current tile (magnitude in its tier)
    uint8_t k[2][kPlane];    // b-tier ping-pong of the current tile (the tier where b > 0, else kKNone)
    uint32_t ks[2][kThreads];  // per thread: the tier summary of its 8 cells (tier_summary)
};

// Tile activity flags (kActB, kActA: common.cuh); kActA tests the encoded A != +0.

template <int kHalo>
__device__ __forceinline__ void tile_origin(int tile, int tiles_x, int& r0, int& c0) {
    constexpr int kIR = kRT - 2 * kHalo, kIC = kCT - 2 * kHalo;
    const int ty = tile / tiles_x, tx = tile % tiles_x;
    r0 = ty * kIR - kHalo;
    c0 = tx * kIC - kHalo;
}

// kRc: q recomputed from the fields of pa (prep's arithmetic, q_cell) for every live
// tile instead of staged from the materialised planes by TMA; the same bits either way.
template <int kHalo, bool kRc>
__global__ void __launch_bounds__(kThreads, 1)
    k_diff_blocked(const __grid_constant__ CUtensorMap tab, const __grid_constant__ CUtensorMap tq,
                   const __grid_constant__ PrepArgs pa, int H, int pitch,
                   int W, float pc, int n, int tiles_x, const int* __restrict__ tiles,
                   const int* __restrict__ ntiles_live, int* __restrict__ work, float* __restrict__ out,
                   float* __restrict__ all_out,
                   size_t all_stride, uint8_t* __restrict__ act_out, unsigned long long* __restrict__ skipped,
                   int* __restrict__ err, TmaHook hk, TileTape tape) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    constexpr int kI = kRT - 2 * kHalo;  // interior side (a tape block is [2][kI][kI])
    const unsigned long long tbase = tape.data ? *tape.used : 0ull;
    __shared__ __align__(8) uint64_t bar;
    // the list index of this CTA's next tile: tiles are handed out dynamically (the first
    // is blockIdx.x, then work counter claims), one tile ahead for the TMA prefetch
    __shared__ int s_next;
    const int tid = threadIdx.x;
    const int x = tid % kCT;             // region column
    const int strip = tid / kCT;
    const int ys = strip * kM;           // first region row of the strip
    const uint32_t bytes = (uint32_t)(((kRc ? 0 : 8) + 2) * kPlane * sizeof(float));
    const size_t gplane = (size_t)H * pitch;

    const int ntiles = *ntiles_live;  // tiles listed by k_fwd_tiles
    int li = blockIdx.x;
    if (li >= ntiles) return;
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        int r0, c0;
        tile_origin<kHalo>(tiles[li], tiles_x, r0, c0);
        mbar_arrive_expect_tx(&bar, bytes);
        if (!hk.withhold) {
            if (!kRc) tma_load_3d(sm.q, &tq, &bar, c0, r0, 0);
            tma_load_3d(sm.st, &tab, &bar, c0, r0, 0);
        }
    }
    uint32_t parity = 0;
    float q[kM][8];
    float A[kM];
    for (;;) {
        const int tile = tiles[li];
        const bool ok = mbar_wait_bounded(&bar, parity, hk.spin);
        if (!__syncthreads_and(ok)) {
            if (tid == 0) {
                atomicExch(err, kErrTmaTimeout);
                mbar_wait_bounded(&bar, parity, hk.spin);
            }
            return;
        }
        parity ^= 1u;
        // stage -> registers (q, A) and -> ping-pong buffer 0 (b and its tier)
        bool burning = false;
        uint32_t kword = 0u;  // this thread's tiers, packed
#pragma unroll
        for (int m = 0; m < kM; ++m) {
            const int y = ys + m;
            if (!kRc)
#pragma unroll
                for (int d = 0; d < 8; ++d) q[m][d] = sm.q[d * kPlane + y * kCT + x];
            float bv;
            int kv;
            x_decode(sm.st[y * kCT + x], sm.st[kPlane + y * kCT + x], A[m], bv, kv);
            sm.b[0][y * kCT + x] = bv;
            sm.k[0][y * kCT + x] = (uint8_t)(bv != 0.0f ? kv : kKNone);
            kword |= (__float_as_uint(A[m]) == 0u ? 15u : (uint32_t)kv) << (4 * m);
            burning |= bv != 0.0f;
        }
        uint32_t ksum = tier_summary(kword);
        sm.ks[0][tid] = ksum;
        fence_proxy_async();  // these generic reads of the stage precede the next TMA writes
        // b = 0 in the whole region: every P is 0 at every step of the launch, so the
        // region's state does not change and the steps are skipped (the stores remain)
        const bool live = __syncthreads_or(burning);  // also: stage fully consumed
        int next = ntiles;
        if (tid == 0) {
            next = (int)gridDim.x + atomicAdd(work, 1);
            s_next = next;  // read by every thread after this tile's last barrier
        }
        if (tid == 0 && next < ntiles) {
            int r0, c0;
            tile_origin<kHalo>(tiles[next], tiles_x, r0, c0);
            mbar_arrive_expect_tx(&bar, bytes);
            if (!hk.withhold) {
                if (!kRc) tma_load_3d(sm.q, &tq, &bar, c0, r0, 0);
                tma_load_3d(sm.st, &tab, &bar, c0, r0, 0);
            }
        }
        int r0, c0;
        tile_origin<kHalo>(tile, tiles_x, r0, c0);
        if (kRc && live) {
            // q of this thread's cells (0 outside the grid, as the TMA fill and the zero
            // padding columns give), through this thread's own slots of sm.q, which no
            // copy writes in this variant
            for (int m = 0; m < kM; ++m) {
                const int y = ys + m, gr = r0 + y, gc = c0 + x;
                float qv[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
                if (gr >= 0 && gr < H && gc >= 0 && gc < W) q_cell(pa, gr, gc, qv);
#pragma unroll
                for (int d = 0; d < 8; ++d) sm.q[d * kPlane + y * kCT + x] = qv[d];
            }
#pragma unroll
            for (int m = 0; m < kM; ++m)
#pragma unroll
                for (int d = 0; d < 8; ++d) q[m][d] = sm.q[d * kPlane + (ys + m) * kCT + x];
        }
        const bool xin = (x >= 1 && x < kCT - 1);
        if (!live && tid == 0 && skipped)
            atomicAdd(skipped, (unsigned long long)(min(kRT - 2 * kHalo, H - (r0 + kHalo)) *
                                                    min(kCT - 2 * kHalo, W - (c0 + kHalo))) *
                                   (unsigned long long)n);
        int cur = 0;
        for (int s = 0; s < n; ++s) {
            if (live) {
                const float* src = sm.b[cur];
                float* dst = sm.b[cur ^ 1];
                const uint8_t* ksrc = sm.k[cur];
                uint8_t* kdst = sm.k[cur ^ 1];
                const int xl = xin ? x - 1 : x, xr = xin ? x + 1 : x;
                // Whether the cells of this thread's windows (rows ys-1 .. ys+8, columns
                // x-1 .. x+1) that are not 0 are all in one tier k0 (from the per-thread tier
                // summaries); when it holds for every lane of the warp, the warp takes the
                // update specialised to one tier (the general one on such inputs, bit for
                // bit), otherwise the general update with per-neighbour tiers.
                uint32_t k0;
                const bool uni = window_one_tier(sm.ks[cur], tid, x - xl, xr - x, strip > 0, strip < kRT / kM - 1,
                                                 kCT, ksum, k0);
                uint32_t knew = kword;
                if (__all_sync(0xffffffffu, uni)) {
                    // one tier k0 for the whole warp (adjacent lanes share window columns)
                    // ring of b rows ys-1 .. ys+kM (slot (row - ys + 1) % 3) in columns x-1, x, x+1
                    float bw[3][3];
                    const int y_first = ys > 0 ? ys - 1 : 0;
                    bw[0][0] = src[y_first * kCT + xl]; bw[0][1] = src[y_first * kCT + x]; bw[0][2] = src[y_first * kCT + xr];
                    bw[1][0] = src[ys * kCT + xl];      bw[1][1] = src[ys * kCT + x];      bw[1][2] = src[ys * kCT + xr];
#pragma unroll
                    for (int m = 0; m < kM; ++m) {
                        const int y = ys + m;
                        float(&bu)[3] = bw[m % 3];
                        float(&bm)[3] = bw[(m + 1) % 3];
                        float(&bd)[3] = bw[(m + 2) % 3];
                        const int yn = y + 1 < kRT ? y + 1 : y;
                        bd[0] = src[yn * kCT + xl]; bd[1] = src[yn * kCT + x]; bd[2] = src[yn * kCT + xr];
                        if (y >= 1 && y < kRT - 1) {  // the region's edge rows are never updated
                            // the edge columns are never updated either: they compute on their
                            // clamped (in-bounds) window like the others and keep their old
                            // values, a select rather than a divergent branch
                            // neighbours in direction order (-1,-1) (-1,0) (-1,1) (0,-1) (0,1) (1,-1) (1,0) (1,1)
                            const float nb[8] = {bu[0], bu[1], bu[2], bm[0], bm[2], bd[0], bd[1], bd[2]};
                            float An, Bn;
                            int kn;
                            if (k0 == 0u) {
                                // tier 0: Eq. 9 with the survival product
                                float P = 0.0f, S = 1.0f;
#pragma unroll
                                for (int d = 0; d < 8; ++d) ign_acc(__fmul_rn(nb[d], q[m][d]), P, S);
                                x_update_t0(P, S, A[m], bm[1], pc, An, Bn, kn);
                            } else {
                                // one tier below 2^-64: every true term is below 2^-61, so the
                                // survival product is 1, 1 - a is 1 and P is a plain sum
                                float P = 0.0f;
#pragma unroll
                                for (int d = 0; d < 8; ++d) P = fmaf(__fmul_rn(nb[d], q[m][d]), 1.0f, P);
                                An = __fadd_rn(A[m], P);
                                Bn = fmaf(pc, bm[1], P);
                                kn = (int)k0;
                                x_renorm(An, Bn, kn);
                            }
                            if (xin) {  // an edge column keeps its cell
                                A[m] = An;
                                dst[y * kCT + x] = Bn;
                                kdst[y * kCT + x] = (uint8_t)(Bn != 0.0f ? kn : kKNone);
                                const uint32_t nib = __float_as_uint(An) == 0u ? 15u : (uint32_t)kn;
                                knew = (knew & ~(15u << (4 * m))) | (nib << (4 * m));
                            } else {
                                dst[y * kCT + x] = bm[1];
                                kdst[y * kCT + x] = ksrc[y * kCT + x];
                            }
                        }
                    }
                } else {
                    // General: per-neighbour tiers. Rolling windows of b and of 64 x the
                    // b-tier over rows ys-1 .. ys+kM in columns x-1, x, x+1 (slot (row - ys + 1)
                    // % 3), and each window row's least b-tier; kP of a cell is the least over
                    // the rows above and below and its own row's left and right cells.
                    float bw[3][3];
                    int tw[3][3], rmin[3];
                    const int cols[3] = {xl, x, xr};
                    const int y_first = ys > 0 ? ys - 1 : 0;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        bw[0][c] = src[y_first * kCT + cols[c]];
                        tw[0][c] = 64 * (int)ksrc[y_first * kCT + cols[c]];
                        bw[1][c] = src[ys * kCT + cols[c]];
                        tw[1][c] = 64 * (int)ksrc[ys * kCT + cols[c]];
                    }
                    rmin[0] = min(min(tw[0][0], tw[0][1]), tw[0][2]);
                    rmin[1] = min(min(tw[1][0], tw[1][1]), tw[1][2]);
#pragma unroll
                    for (int m = 0; m < kM; ++m) {
                        const int y = ys + m;
                        const int su = m % 3, sc = (m + 1) % 3, sd = (m + 2) % 3;
                        const int yn = y + 1 < kRT ? y + 1 : y;
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            bw[sd][c] = src[yn * kCT + cols[c]];
                            tw[sd][c] = 64 * (int)ksrc[yn * kCT + cols[c]];
                        }
                        rmin[sd] = min(min(tw[sd][0], tw[sd][1]), tw[sd][2]);
                        if (y >= 1 && y < kRT - 1) {
                            // the edge columns compute on their clamped window and keep their
                            // old values, as in the path above
                            const int kP64 = min(min(rmin[su], rmin[sd]), min(tw[sc][0], tw[sc][2]));
                            const int e0 = 127 + kP64;  // tier_scale(t - kP) = 2^(e0 - 64 t - 127) or 0
                            const bool kP0 = kP64 == 0;
                            const float nb[8] = {bw[su][0], bw[su][1], bw[su][2], bw[sc][0], bw[sc][2], bw[sd][0], bw[sd][1], bw[sd][2]};
                            const int nt[8] = {tw[su][0], tw[su][1], tw[su][2], tw[sc][0], tw[sc][2], tw[sd][0], tw[sd][1], tw[sd][2]};
                            float P = 0.0f, S = 1.0f;
#pragma unroll
                            for (int d = 0; d < 8; ++d) {
                                const float f = __int_as_float(max(e0 - nt[d], 0) << 23);
                                const float xx = __fmul_rn(__fmul_rn(nb[d], q[m][d]), f);
                                P = fmaf(xx, S, P);
                                S = kP0 ? fmaf(-xx, S, S) : S;
                            }
                            const uint32_t nib = (kword >> (4 * m)) & 15u;
                            float An, Bn;
                            int kn;
                            x_own(P, S, kP64 >> 6, A[m], bw[sc][1], nib == 15u ? 0 : (int)nib, pc, An, Bn, kn);
                            if (xin) {
                                A[m] = An;
                                dst[y * kCT + x] = Bn;
                                kdst[y * kCT + x] = (uint8_t)(Bn != 0.0f ? kn : kKNone);
                                const uint32_t nn = __float_as_uint(An) == 0u ? 15u : (uint32_t)kn;
                                knew = (knew & ~(15u << (4 * m))) | (nn << (4 * m));
                            } else {
                                dst[y * kCT + x] = bw[sc][1];
                                kdst[y * kCT + x] = ksrc[y * kCT + x];
                            }
                        }
                    }
                }
                kword = knew;
                ksum = tier_summary(kword);
                sm.ks[cur ^ 1][tid] = ksum;
                __syncthreads();
                cur ^= 1;
            }
            if (all_out) {  // every intermediate state (segment recompute for the adjoint)
                float* o = all_out + (size_t)s * all_stride;
                const int gc = c0 + x;
                if (x >= kHalo && x < kCT - kHalo && gc < pitch) {
#pragma unroll
                    for (int m = 0; m < kM; ++m) {
                        const int y = ys + m, gr = r0 + y;
                        if (y >= kHalo && y < kRT - kHalo && gr < H) {
                            float As, Bs;
                            const uint32_t nib = (kword >> (4 * m)) & 15u;
                            x_encode(A[m], sm.b[cur][y * kCT + x], nib == 15u ? 0 : (int)nib, As, Bs);
                            o[(size_t)gr * pitch + gc] = As;
                            o[gplane + (size_t)gr * pitch + gc] = Bs;
                        }
                    }
                }
            }
            if (tape.data) {  // the tile tape: this state of a live tile as a block
                const unsigned long long blk = tbase + (unsigned long long)li * n + s;
                const int gc = c0 + x;
                if (blk < tape.cap && x >= kHalo && x < kCT - kHalo && gc < pitch) {
                    float* o = tape.data + blk * (2ull * kI * kI);
#pragma unroll
                    for (int m = 0; m < kM; ++m) {
                        const int y = ys + m, gr = r0 + y;
                        if (y >= kHalo && y < kRT - kHalo && gr < H) {
                            float As, Bs;
                            const uint32_t nib = (kword >> (4 * m)) & 15u;
                            x_encode(A[m], sm.b[cur][y * kCT + x], nib == 15u ? 0 : (int)nib, As, Bs);
                            const int o_ = (y - kHalo) * kI + (x - kHalo);
                            o[o_] = As;
                            o[kI * kI + o_] = Bs;
                        }
                    }
                }
            }
        }
        if (out) {
            const int gc = c0 + x;
            if (x >= kHalo && x < kCT - kHalo && gc < pitch) {
#pragma unroll
                for (int m = 0; m < kM; ++m) {
                    const int y = ys + m, gr = r0 + y;
                    if (y >= kHalo && y < kRT - kHalo && gr < H) {
                        float As, Bs;
                        const uint32_t nib = (kword >> (4 * m)) & 15u;
                        x_encode(A[m], sm.b[cur][y * kCT + x], nib == 15u ? 0 : (int)nib, As, Bs);
                        out[(size_t)gr * pitch + gc] = As;
                        out[gplane + (size_t)gr * pitch + gc] = Bs;
                    }
                }
            }
        }
        // whether b > 0 anywhere in the interior after the launch (for the next launch's
        // tile list); the barrier also protects the ping-pong buffers reused by the next tile
        bool actB = false, actA = false;
        if (x >= kHalo && x < kCT - kHalo) {
#pragma unroll
            for (int m = 0; m < kM; ++m) {
                const int y = ys + m;
                if (y >= kHalo && y < kRT - kHalo) {
                    actB |= sm.b[cur][y * kCT + x] != 0.0f;
                    actA |= __float_as_uint(A[m]) != 0u;
                }
            }
        }
        actB = __syncthreads_or(actB);
        actA = __syncthreads_or(actA);
        if (tid == 0) act_out[tile] = (act_out[tile] & kQb) | (actA ? kActA : 0) | (actB ? kActB : 0);
        li = s_next;
        if (li >= ntiles) break;
    }
}

// Activity of a state at the start of a chain of launches; qrun[tile] = 0 (nothing is
// known about the other buffers). One warp per tile.
template <int kHalo>
__global__ void __launch_bounds__(256) k_fwd_act_init(const float* __restrict__ ab, int H, int pitch, int tiles_x,
                                                      int ntiles, uint8_t* __restrict__ act,
                                                      uint8_t* __restrict__ qrun) {
    constexpr int kI = kRT - 2 * kHalo;
    const int tile = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (tile >= ntiles) return;
    int r0, c0;
    tile_origin<kHalo>(tile, tiles_x, r0, c0);
    r0 += kHalo;
    c0 += kHalo;
    const size_t gplane = (size_t)H * pitch;
    uint32_t anyA = 0u, anyB = 0u;
    // float4 columns: c0 and pitch are multiples of 4
    for (int i = lane; i < kI * (kI / 4); i += 32) {
        const int gr = r0 + i / (kI / 4), gc = c0 + 4 * (i % (kI / 4));
        if (gr >= H || gc >= pitch) continue;
        const uint4 a = __ldg(reinterpret_cast<const uint4*>(ab + (size_t)gr * pitch + gc));
        const uint4 b = __ldg(reinterpret_cast<const uint4*>(ab + gplane + (size_t)gr * pitch + gc));
        anyA |= a.x | a.y | a.z | a.w;
        anyB |= (b.x | b.y | b.z | b.w) & 0x7fffffffu;
    }
    const bool hasA = __any_sync(0xffffffffu, anyA != 0u), hasB = __any_sync(0xffffffffu, anyB != 0u);
    if (lane == 0) {
        act[tile] = (hasA ? kActA : 0) | (hasB ? kActB : 0) | kQt;  // nothing happened yet
        qrun[tile] = 0;
    }
}

// The same from flags recorded for the state by an earlier chain (its launch's act_out):
// their activity bits are exact, the segment bits start afresh.
__global__ void __launch_bounds__(256) k_fwd_act_seed(const uint8_t* __restrict__ seed, int ntiles,
                                                      uint8_t* __restrict__ act, uint8_t* __restrict__ qrun) {
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= ntiles) return;
    act[i] = (uint8_t)((seed[i] & (kActA | kActB)) | kQt);
    qrun[i] = 0;
}

// Pre-pass of one forward launch, one warp per tile. A tile is live if b > 0 anywhere in
// the interiors of the 3 x 3 tiles around it (act_in, from the previous launch or
// k_fwd_act_init): its region (interior + halo <= one interior) lies inside them, so a
// tile that is not live has b = 0 in its whole region and its state does not change
// during the launch. Live tiles are listed for k_diff_blocked, which writes their
// act_out. A quiescent tile keeps its kActA flag; its interior is copied to the outputs,
// except into `out` when out already holds its state: out holds the input state of the
// launch out_age launches back (out_age > 0) and the tile has been quiescent in every
// launch since (qrun[tile], the tile's quiescent streak, saturating at 255).
//
// Segment buffers (seg_rng != nullptr): all_out is a run of slots of a buffer that is
// reused from segment to segment (slot_a .. slot_a + n - 1 counted from zero_base), and
// seg_rng[tile] = lo | hi << 16 bounds the slots [lo, hi) where the tile's interior may
// be nonzero. A quiescent tile with a = 0 in the 3 x 3 interiors around it is void
// (exactly zero in its whole region for the whole launch); the launch's slots only have
// to hold zeros there, which they already do outside the range. The launch zeroes its
// own slots inside it, and the range loses them when they are its front: the launches of
// a segment run in slot order, so a tile that turns live within a segment zeroes only the
// slots before, and in the segment after (earlier in time) only the rest.
//
// Aligned segment recompute (frozen != 0): quiescent tiles get kFrozen (their region is
// constant over the launch). One with b = 0 in the 5 x 5 interiors around it writes only
// the launch's last slot (the next launch's input): every tile whose region reaches into
// it is frozen too and is read at its first slot only. One with b = 0 in the 7 x 7
// interiors whose 5 x 5 tiles have all been quiescent since the segment's start (kQt)
// writes nothing and is marked kStale. Then every tile whose region reaches into it is
// quiescent in this launch and the next, and kQb (unchanged since slot 0) in the next.
// So the adjoint reads those tiles' regions from slot0 (kTileCkptBit), which holds the
// stale tile's state, and no live tile's region reaches it before it writes again. When
// it does, it copies from slot0.
template <int kHalo>
__device__ __forceinline__ void fwd_tile(const float* __restrict__ in, int H, int W, int pitch,
                                                   int tiles_x, int tiles_y, int n, const uint8_t* __restrict__ act_in,
                                                   uint8_t* __restrict__ act_out, uint8_t* __restrict__ qrun,
                                                   int* __restrict__ list, int* __restrict__ count,
                                                   float* __restrict__ out, int out_age,
                                                   float* __restrict__ all_out, size_t all_stride,
                                                   uint32_t* __restrict__ seg_rng, const float* __restrict__ slot0,
                                                   float* __restrict__ zero_base, int slot_a, int frozen,
                                                   uint8_t* __restrict__ out_dirty, int dirty_unknown,
                                                   unsigned long long* __restrict__ skipped, int tile, int lane,
                                                   unsigned long long& sk, unsigned long long& wr) {
    constexpr int kI = kRT - 2 * kHalo;
    const int ty = tile / tiles_x, tx = tile % tiles_x;
    // the tile's own entries, loaded with the flags below so that their latencies overlap
    // (each is read before this warp writes it, and no other warp touches them)
    const uint32_t me = act_in[tile];
    const int qr = qrun[tile];
    const uint32_t rng = seg_rng ? seg_rng[tile] : 0u;
    const bool od = out_dirty ? out_dirty[tile] != 0 : false;
    // the 7 x 7 flags around the tile, two per lane (independent loads), reduced into the
    // ORs over the 3 x 3, 5 x 5 and 7 x 7 tiles and the AND of kQt over the 5 x 5 (tiles
    // outside the grid count as quiescent and empty)
    uint32_t o3 = 0u, o5 = 0u, o7 = 0u, q5 = 1u;
    for (int p = lane; p < 49; p += 32) {
        const int dy = p / 7 - 3, dx = p % 7 - 3;
        const int yy = ty + dy, xx = tx + dx;
        const bool in_grid = yy >= 0 && yy < tiles_y && xx >= 0 && xx < tiles_x;
        const uint32_t f = in_grid ? act_in[yy * tiles_x + xx] : 0u;
        o7 |= f;
        if (dy >= -2 && dy <= 2 && dx >= -2 && dx <= 2) {
            o5 |= f;
            if (in_grid && !(f & kQt)) q5 = 0u;
        }
        if (dy >= -1 && dy <= 1 && dx >= -1 && dx <= 1) o3 |= f;
    }
    const uint32_t around = __reduce_or_sync(0xffffffffu, o3);
    const uint32_t around5 = __reduce_or_sync(0xffffffffu, o5);
    const uint32_t around7 = __reduce_or_sync(0xffffffffu, o7);
    const bool qseg5 = __reduce_and_sync(0xffffffffu, q5) != 0u;
    const uint8_t qb = (me & kQt) ? kQb : 0;  // quiescent in every earlier launch of the segment
    // the tile's dirty slot range grows by [w0, slot_a + n) (lane 0)
    auto rng_add = [&](int w0) {
        const uint32_t r = rng;
        int lo = (int)(r & 0xffffu), hi = (int)(r >> 16);
        if (lo >= hi) lo = w0, hi = slot_a + n;
        else lo = min(lo, w0), hi = max(hi, slot_a + n);
        seg_rng[tile] = (uint32_t)lo | ((uint32_t)hi << 16);
    };
    if (around & kActB) {
        if (lane == 0) {
            list[atomicAdd(count, 1)] = tile;
            qrun[tile] = 0;
            if (seg_rng) rng_add(slot_a);
            if (out_dirty) out_dirty[tile] = 1;
            act_out[tile] = qb;  // k_diff_blocked adds the tile's activity
        }
        return;
    }
    const int r0 = ty * kI, c0 = tx * kI;
    const size_t gplane = (size_t)H * pitch;
    bool write_all = all_out != nullptr;
    const bool void_tile = seg_rng && !(around & kActA);
    if (void_tile) {
        write_all = false;
        const int lo = (int)(rng & 0xffffu), hi = (int)(rng >> 16);
        const int z0 = max(lo, slot_a), z1 = min(hi, slot_a + n);
        if (z0 < z1) {
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int i = lane; i < kI * (kI / 4); i += 32) {
                const int gr = r0 + i / (kI / 4), gc = c0 + 4 * (i % (kI / 4));
                if (gr >= H || gc >= pitch) continue;
                const size_t j = (size_t)gr * pitch + gc;
                for (int s = z0; s < z1; ++s) {
                    float* o = zero_base + (size_t)s * all_stride;
                    *reinterpret_cast<float4*>(o + j) = z;
                    *reinterpret_cast<float4*>(o + gplane + j) = z;
                }
            }
            __syncwarp();
            if (lane == 0) {
                if (z0 == lo) seg_rng[tile] = z1 >= hi ? 0u : ((uint32_t)z1 | ((uint32_t)hi << 16));
                wr += (unsigned long long)(min(kI, H - r0) * min(kI, W - c0)) * (unsigned long long)(z1 - z0);
            }
        }
    }
    // far from anything burning: only the last slot (the next launch's input) is read;
    // farther still and unchanged since slot 0 around it: nothing is
    const bool last_only = frozen && write_all && !(around5 & kActB);
    const bool stale = last_only && slot0 && !(around7 & kActB) && qseg5;
    if (stale) write_all = false;
    // a tile that skipped its last write takes its state from slot 0
    const float* src = (frozen && slot0 && (me & kStale)) ? slot0 : in;
    bool copy_out = out && !(out_age > 0 && qr >= out_age);
    // a checkpoint slot with dirty bits (out_dirty): an all-zero tile (a = 0 in the
    // interior, so b = 0 too) is written only if the slot's tile may hold nonzeros
    bool zero_out = false;
    if (copy_out && out_dirty && !(me & kActA)) {
        zero_out = dirty_unknown || od;
        copy_out = false;
    }
    if (zero_out) {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i = lane; i < kI * (kI / 4); i += 32) {
            const int gr = r0 + i / (kI / 4), gc = c0 + 4 * (i % (kI / 4));
            if (gr >= H || gc >= pitch) continue;
            const size_t j = (size_t)gr * pitch + gc;
            *reinterpret_cast<float4*>(out + j) = z;
            *reinterpret_cast<float4*>(out + gplane + j) = z;
        }
    }
    // In an aligned recompute the tile is frozen in the matching adjoint launch, which
    // reads its region from the launch's first state only; the other tiles' regions reach
    // 8 cells into its interior. So slots before the last need only that 8-cell band, and
    // the last slot (the next launch's input) the whole interior.
    const bool band_only = frozen && seg_rng;
    if (seg_rng && write_all && lane == 0) rng_add(last_only ? slot_a + n - 1 : slot_a);
    uint32_t nw = 0u;  // float4 pairs this lane wrote
    if (copy_out || write_all) {
        // float4 columns: c0 and pitch are multiples of 4 (and 8, kI - 8 are too). Each
        // lane loads kU float4 pairs before it stores any, so their latencies overlap.
        constexpr int kPer = kI * (kI / 4);
        constexpr int kU = 2;
        for (int i0 = lane; i0 < kPer; i0 += 32 * kU) {
            float4 a[kU], b[kU];
            size_t jj[kU];
            bool ok[kU], band[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int i = i0 + 32 * u;
                const int ir = i / (kI / 4), ic = 4 * (i % (kI / 4));
                const int gr = r0 + ir, gc = c0 + ic;
                ok[u] = i < kPer && gr < H && gc < pitch;
                band[u] = ir < 8 || ir >= kI - 8 || ic < 8 || ic >= kI - 8;
                jj[u] = (size_t)gr * pitch + gc;
                if (ok[u]) {
                    a[u] = __ldg(reinterpret_cast<const float4*>(src + jj[u]));
                    b[u] = __ldg(reinterpret_cast<const float4*>(src + gplane + jj[u]));
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                if (!ok[u]) continue;
                const size_t j = jj[u];
                if (copy_out) {
                    *reinterpret_cast<float4*>(out + j) = a[u];
                    *reinterpret_cast<float4*>(out + gplane + j) = b[u];
                    ++nw;
                }
                if (write_all) {
                    for (int s = last_only ? n - 1 : 0; s < n; ++s) {
                        if (band_only && s < n - 1 && !band[u]) continue;
                        float* o = all_out + (size_t)s * all_stride;
                        *reinterpret_cast<float4*>(o + j) = a[u];
                        *reinterpret_cast<float4*>(o + gplane + j) = b[u];
                        ++nw;
                    }
                }
            }
        }
    }
    nw = __reduce_add_sync(0xffffffffu, nw);
    __syncwarp();  // qrun[tile] read by every lane before it changes
    if (lane == 0) {
        if (out_dirty && out) out_dirty[tile] = (me & kActA) ? 1 : 0;
        act_out[tile] = (uint8_t)((me & (kActA | kQt)) | qb | (frozen ? kFrozen : 0) | (stale ? kStale : 0));
        qrun[tile] = (uint8_t)min(qr + 1, 255);
        sk = (unsigned long long)(min(kI, H - r0) * min(kI, W - c0)) * (unsigned long long)n;
        // cells this pre-pass wrote into its output buffers (copies and zero fills)
        wr += 4ull * nw + (zero_out ? (unsigned long long)(min(kI, H - r0) * min(kI, W - c0)) : 0ull);
    }
}

template <int kHalo>
__global__ void __launch_bounds__(256, 5) k_fwd_tiles(const float* __restrict__ in, int H, int W, int pitch,
                                                   int tiles_x, int tiles_y, int n, const uint8_t* __restrict__ act_in,
                                                   uint8_t* __restrict__ act_out, uint8_t* __restrict__ qrun,
                                                   int* __restrict__ list, int* __restrict__ count,
                                                   float* __restrict__ out, int out_age,
                                                   float* __restrict__ all_out, size_t all_stride,
                                                   uint32_t* __restrict__ seg_rng, const float* __restrict__ slot0,
                                                   float* __restrict__ zero_base, int slot_a, int frozen,
                                                   uint8_t* __restrict__ out_dirty, int dirty_unknown,
                                                   unsigned long long* __restrict__ skipped,
                                                   unsigned long long* __restrict__ written) {
    __shared__ unsigned long long s_sk, s_wr;
    if (threadIdx.x == 0) s_sk = s_wr = 0ull;
    __syncthreads();
    unsigned long long sk = 0ull, wr = 0ull;
    const int tile = blockIdx.x * 8 + (threadIdx.x >> 5);  // one warp per tile
    if (tile < tiles_x * tiles_y)
        fwd_tile<kHalo>(in, H, W, pitch, tiles_x, tiles_y, n, act_in, act_out, qrun, list, count, out,
                        out_age, all_out, all_stride, seg_rng, slot0, zero_base, slot_a, frozen, out_dirty,
                        dirty_unknown, skipped, tile, threadIdx.x & 31, sk, wr);
    block_count(skipped, s_sk, sk);
    block_count(written, s_wr, wr);
}

// After a taped launch (one block of 256 threads): the launch's record and list.
__global__ void __launch_bounds__(256) k_tape_record(TileTape tape, const int* __restrict__ tile_count,
                                                     const int* __restrict__ tile_list, int n, int L,
                                                     unsigned long long* __restrict__ meta, int* __restrict__ lists,
                                                     int list_cap) {
    const unsigned long long count = (unsigned long long)*tile_count;
    const unsigned long long base = *tape.used;
    const bool ok = base + count * (unsigned long long)n <= tape.cap;
    __syncthreads();  // every thread has read tape.used before thread 0 advances it
    if (threadIdx.x == 0) {
        meta[4 * L + 0] = base;
        meta[4 * L + 1] = (unsigned long long)n;
        meta[4 * L + 2] = count;
        meta[4 * L + 3] = ok ? 1ull : 0ull;
        if (ok) *tape.used = base + count * (unsigned long long)n;
    }
    if (ok)
        for (unsigned long long i = threadIdx.x; i < count; i += 256) lists[(size_t)L * list_cap + i] = tile_list[i];
}

// inv[tile] = its index in a record's list (inv holds -1 elsewhere)
__global__ void __launch_bounds__(256) k_tape_inv(const int* __restrict__ rec_list, int rec_count,
                                                  int* __restrict__ inv) {
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i < rec_count) inv[rec_list[i]] = i;
}

// Work item w = (entry w / n of the recompute's list, step w % n), taken by the blocks
// in turn (grid-stride): the tile's state at that step from the tape into its segment
// slot; the last step's item also writes the tile's activity after the launch (as
// k_diff_blocked writes it).
template <int kHalo>
__global__ void __launch_bounds__(256) k_tape_unpack(const float* __restrict__ tape_data, unsigned long long base,
                                                     int n_rec, const int* __restrict__ inv,
                                                     const int* __restrict__ tile_list,
                                                     const int* __restrict__ tile_count, int n, int H, int pitch,
                                                     int tiles_x, float* __restrict__ all_out, size_t all_stride,
                                                     uint8_t* __restrict__ act_out, int* __restrict__ missing) {
    constexpr int kI = kRT - 2 * kHalo;
    constexpr int kPer = kI * (kI / 4);             // float4 of a plane
    constexpr int kU = (kPer + 255) / 256;          // of them a thread
    __shared__ int s_any[2];
    const int items = *tile_count * n;
    const size_t gplane = (size_t)H * pitch;
    for (int w = blockIdx.x; w < items; w += gridDim.x) {  // uniform across the block
        const int st = w % n;
        const int tile = tile_list[w / n];
        const int li = inv[tile];
        if (li < 0) {  // not in the record: the caller recomputes the segment
            if (threadIdx.x == 0 && st == 0) atomicAdd(missing, 1);
            continue;
        }
        const bool last = st == n - 1;
        if (last && threadIdx.x == 0) s_any[0] = s_any[1] = 0;
        const int ty = tile / tiles_x, tx = tile % tiles_x;
        const int r0 = ty * kI, c0 = tx * kI;
        const float* src = tape_data + (base + (unsigned long long)li * n_rec + st) * (2ull * kI * kI);
        float* o = all_out + (size_t)st * all_stride;
        // every load of the thread before any store; float4 columns (c0 and pitch are
        // multiples of 4)
        float4 a[kU], b[kU];
        size_t jo[kU];
        bool ok[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int i = threadIdx.x + 256 * u;
            const int ir = i / (kI / 4), ic = 4 * (i % (kI / 4));
            const int gr = r0 + ir, gc = c0 + ic;
            ok[u] = i < kPer && gr < H && gc < pitch;
            jo[u] = (size_t)gr * pitch + gc;
            if (ok[u]) {
                a[u] = *reinterpret_cast<const float4*>(src + ir * kI + ic);
                b[u] = *reinterpret_cast<const float4*>(src + kI * kI + ir * kI + ic);
            }
        }
        int anyA = 0, anyB = 0;
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (!ok[u]) continue;
            *reinterpret_cast<float4*>(o + jo[u]) = a[u];
            *reinterpret_cast<float4*>(o + gplane + jo[u]) = b[u];
            anyA |= (__float_as_uint(a[u].x) | __float_as_uint(a[u].y) | __float_as_uint(a[u].z) |
                     __float_as_uint(a[u].w)) != 0u;
            anyB |= b[u].x != 0.0f || b[u].y != 0.0f || b[u].z != 0.0f || b[u].w != 0.0f;
        }
        if (!last) continue;
        __syncthreads();  // s_any cleared
        if (anyA) s_any[0] = 1;
        if (anyB) s_any[1] = 1;
        __syncthreads();
        if (threadIdx.x == 0)
            act_out[tile] = (uint8_t)((act_out[tile] & kQb) | (s_any[0] ? kActA : 0) | (s_any[1] ? kActB : 0));
    }
}

}  // namespace

int diff_blocked_halo() { return kHaloMax; }
int diff_blocked_box_rows() { return kRT; }
int diff_blocked_box_cols() { return kCT; }

size_t diff_blocked_smem() { return sizeof(Smem) + 128; }

int diff_blocked_configure() {
    static int done = 0;
    if (!done) {
        if (cudaFuncSetAttribute(k_diff_blocked<8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)diff_blocked_smem()) != cudaSuccess ||
            cudaFuncSetAttribute(k_diff_blocked<4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)diff_blocked_smem()) != cudaSuccess ||
            cudaFuncSetAttribute(k_diff_blocked<8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)diff_blocked_smem()) != cudaSuccess ||
            cudaFuncSetAttribute(k_diff_blocked<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)diff_blocked_smem()) != cudaSuccess)
            return -1;
        done = 1;
    }
    return 0;
}

int diff_blocked_tiles(int halo, int H, int pitch) {
    const int inner = kRT - 2 * halo;
    return ((pitch + inner - 1) / inner) * ((H + inner - 1) / inner);
}

void launch_fwd_act_init(int halo, const float* ab, int H, int pitch, uint8_t* act, uint8_t* qrun,
                         cudaStream_t s) {
    const int inner = kRT - 2 * halo;
    const int tiles_x = (pitch + inner - 1) / inner;
    const int ntiles = diff_blocked_tiles(halo, H, pitch);
    const int blocks = (ntiles + 7) / 8;  // one warp per tile
    if (halo == 4)
        k_fwd_act_init<4><<<blocks, 256, 0, s>>>(ab, H, pitch, tiles_x, ntiles, act, qrun);
    else
        k_fwd_act_init<8><<<blocks, 256, 0, s>>>(ab, H, pitch, tiles_x, ntiles, act, qrun);
}

void launch_fwd_act_seed(int halo, const uint8_t* seed, int H, int pitch, uint8_t* act, uint8_t* qrun,
                         cudaStream_t s) {
    const int ntiles = diff_blocked_tiles(halo, H, pitch);
    k_fwd_act_seed<<<(ntiles + 255) / 256, 256, 0, s>>>(seed, ntiles, act, qrun);
}

bool launch_fwd_tiles(int halo, const float* in, int H, int W, int pitch, int n, const uint8_t* act_in,
                      uint8_t* act_out, uint8_t* qrun, int* tile_list, int* tile_count, float* out,
                      int out_age, float* all_out, size_t all_stride, uint32_t* seg_rng, const float* slot0,
                      float* zero_base, int zero_slots, bool frozen, uint8_t* out_dirty, bool dirty_unknown,
                      unsigned long long* skipped, unsigned long long* written, cudaStream_t s) {
    const int inner = kRT - 2 * halo;
    // the launch's first slot, counted from zero_base (slots zero_base .. + zero_slots - 1)
    int slot_a = 0;
    if (seg_rng) {
        slot_a = (int)((all_out - zero_base) / (ptrdiff_t)all_stride);
        if (all_out < zero_base || slot_a + n > zero_slots || slot_a + n > 0xffff) return false;
    }
    const int tiles_x = (pitch + inner - 1) / inner;
    const int tiles_y = (H + inner - 1) / inner;
    cudaMemsetAsync(tile_count, 0, 2 * sizeof(int), s);  // the count and k_diff_blocked's work counter
    if (halo == 4)
        k_fwd_tiles<4><<<(tiles_x * tiles_y + 7) / 8, 256, 0, s>>>(in, H, W, pitch, tiles_x, tiles_y, n, act_in, act_out,
                                                         qrun, tile_list, tile_count, out, out_age,
                                                         all_out, all_stride, seg_rng, slot0, zero_base, slot_a,
                                                         frozen ? 1 : 0, out_dirty, dirty_unknown ? 1 : 0, skipped,
                                                         written);
    else
        k_fwd_tiles<8><<<(tiles_x * tiles_y + 7) / 8, 256, 0, s>>>(in, H, W, pitch, tiles_x, tiles_y, n, act_in, act_out,
                                                         qrun, tile_list, tile_count, out, out_age,
                                                         all_out, all_stride, seg_rng, slot0, zero_base, slot_a,
                                                         frozen ? 1 : 0, out_dirty, dirty_unknown ? 1 : 0, skipped,
                                                         written);
    return true;
}

void launch_diff_blocked(int halo, const CUtensorMap* tab, const CUtensorMap* tq, const PrepArgs* pa, int H, int W,
                         int pitch, float pc, int n, const int* tile_list, int* tile_count, float* out, float* all_out,
                         size_t all_stride, uint8_t* act_out, unsigned long long* skipped, int nsm, int* err,
                         TmaHook hk, TileTape tape, cudaStream_t s) {
    const int inner = kRT - 2 * halo;
    const int tiles_x = (pitch + inner - 1) / inner;
    const int ntiles = diff_blocked_tiles(halo, H, pitch);
    const int grid = ntiles < nsm ? ntiles : nsm;
    const PrepArgs g = pa ? *pa : PrepArgs{};
#define PF_DIFF_BLOCKED(HALO, RC)                                                                                   \
    k_diff_blocked<HALO, RC><<<grid, kThreads, diff_blocked_smem(), s>>>(*tab, *tq, g, H, pitch, W, pc, n, tiles_x, \
                                                                          tile_list, tile_count, tile_count + 1, out, \
                                                                          all_out, all_stride, act_out, skipped, err, hk, \
                                                                          tape)
    if (halo == 4) {
        if (pa) PF_DIFF_BLOCKED(4, true); else PF_DIFF_BLOCKED(4, false);
    } else {
        if (pa) PF_DIFF_BLOCKED(8, true); else PF_DIFF_BLOCKED(8, false);
    }
#undef PF_DIFF_BLOCKED
}

}  // namespace pf

namespace pf {

void launch_tape_record(TileTape tape, const int* tile_count, const int* tile_list, int n, int L,
                        unsigned long long* meta, int* lists, int list_cap, cudaStream_t s) {
    k_tape_record<<<1, 256, 0, s>>>(tape, tile_count, tile_list, n, L, meta, lists, list_cap);
}

void launch_tape_unpack(int halo, const float* tape_data, unsigned long long base, int n_rec, int rec_count,
                        const int* rec_list, int* inv, int ntiles, const int* tile_list, const int* tile_count,
                        int n, int H, int pitch, float* all_out, size_t all_stride, uint8_t* act_out, int* missing,
                        int nsm, cudaStream_t s) {
    if (n <= 0 || ntiles <= 0) return;
    const int inner = kRT - 2 * halo;
    const int tiles_x = (pitch + inner - 1) / inner;
    cudaMemsetAsync(inv, 0xff, sizeof(int) * (size_t)ntiles, s);
    if (rec_count > 0) k_tape_inv<<<(rec_count + 255) / 256, 256, 0, s>>>(rec_list, rec_count, inv);
    // eight blocks an SM (their resident limit) take the items in turn
    const int grid = std::max(1, std::min(ntiles * n, 8 * std::max(nsm, 1)));
    if (halo == 4)
        k_tape_unpack<4><<<grid, 256, 0, s>>>(tape_data, base, n_rec, inv, tile_list, tile_count, n, H, pitch,
                                                tiles_x, all_out, all_stride, act_out, missing);
    else
        k_tape_unpack<8><<<grid, 256, 0, s>>>(tape_data, base, n_rec, inv, tile_list, tile_count, n, H, pitch,
                                                tiles_x, all_out, all_stride, act_out, missing);
}

}  // namespace pf
