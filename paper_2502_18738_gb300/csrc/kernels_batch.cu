// Batched fires: one persistent kernel steps many independent fires of uneven size and
// step count from a device work queue.
//
// A work item is (fire, tile, block b): advance one 32 x 64-cell interior tile of one fire
// by up to kB steps (global steps b*kB ..), reading the tile plus a kB-cell halo from the
// fire's state buffer b % 2 and writing the interior to buffer (b+1) % 2 (or, for the
// fire's last block, to its output). Items are handed out by one atomic counter in
// block-major order (every fire's block b before any block b+1), and an item starts
// only once the 3 x 3 neighbouring tiles have published generation >= b, which also
// guarantees they have finished reading the buffer it overwrites. Because an item waits
// only on items handed out before it, the earliest unfinished item never waits, so the
// queue always drains, whatever number of CTAs is resident. Every wait is bounded in time (globaltimer): on
// timeout the CTA records an error and every CTA stops taking work.
#include "common.cuh"

namespace pf {

// BatchJobDev / BatchPlan (common.cuh): per-fire buffers and the item decoding tables:
// jobs sorted by block count, descending; blk_start[b] = first item of block b;
// tile_pref[j] = tiles of jobs 0 .. j-1; jobs_in_blk[b] = jobs with more than b blocks.

namespace {

constexpr int kB = 4;               // steps per item (= halo)
constexpr int kTR = 32, kTC = 64;   // interior rows / columns
constexpr int kRR = kTR + 2 * kB;   // 40 region rows
constexpr int kRC = kTC + 2 * kB;   // 72 region columns
constexpr int kBThreads = 256;
constexpr int kErrBatchTimeout = 2;  // a wait for a neighbouring tile ran out

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int upper_bound_ll(const long long* a, int n, long long v) {
    int lo = 0, hi = n;  // first index with a[idx] > v
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] > v) hi = mid; else lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ uint8_t disc_update(uint8_t s, const uint8_t* nb, const BatchJobDev& J, const float* q,
                                               size_t qplane, size_t qoff, uint32_t cell, uint32_t step) {
    if (s == 1) {
        float P = 0.0f;
        bool any = false;
#pragma unroll
        for (int d = 0; d < 8; ++d)
            if (nb[d] == 2) {
                any = true;
                const float x = __ldg(q + d * qplane + qoff);
                P = fmaf(x, 1.0f - P, P);
            }
        if (!any) return 1;
        const U4 r = philox10(cell, J.run, step, J.fire, J.key0, J.key1);
        return u24(r.x) < P ? 2 : 1;
    }
    if (s == 2) {
        const U4 r = philox10(cell, J.run, step, J.fire, J.key0, J.key1);
        return u24(r.y) < J.pc ? 2 : 3;
    }
    return s;
}

__global__ void __launch_bounds__(kBThreads) k_batch(BatchPlan plan) {
    __shared__ float sA[2][kRR][kRC];
    __shared__ float sB[2][kRR][kRC];
    __shared__ long long s_item;
    __shared__ int s_ok;
    uint8_t(&s8)[2][kRR][kRC * 4] = *reinterpret_cast<uint8_t(*)[2][kRR][kRC * 4]>(&sA);  // discrete reuse
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) {
            s_item = (*(volatile int*)plan.err) ? plan.total : (long long)atomicAdd(plan.counter, 1ull);
        }
        __syncthreads();
        const long long item = s_item;
        if (item >= plan.total) return;
        // decode (block, job, tile)
        const int b = upper_bound_ll(plan.blk_start, plan.max_blk + 1, item) - 1;
        const long long r = item - plan.blk_start[b];
        const int j = upper_bound_ll(plan.tile_pref, plan.jobs_in_blk[b] + 1, r) - 1;
        const int tile = (int)(r - plan.tile_pref[j]);
        const BatchJobDev& J = plan.jobs[j];
        const int ty = tile / J.tiles_x, tx = tile % J.tiles_x;
        const int r0 = ty * kTR - kB, c0 = tx * kTC - kB;
        // wait until the 3 x 3 neighbourhood has completed block b - 1
        if (tid == 0) {
            int ok = 1;
            for (int dy = -1; dy <= 1 && ok; ++dy)
                for (int dx = -1; dx <= 1 && ok; ++dx) {
                    const int yy = ty + dy, xx = tx + dx;
                    if (yy < 0 || yy >= J.tiles_y || xx < 0 || xx >= J.tiles_x) continue;
                    const volatile int* g = J.gen + yy * J.tiles_x + xx;
                    if (*g >= b) continue;
                    const unsigned long long t0 = global_ns();
                    while (*g < b) {
                        if (global_ns() - t0 > (unsigned long long)plan.wait_limit_ns || *(volatile int*)plan.err) {
                            ok = 0;
                            break;
                        }
                        __nanosleep(100);
                    }
                }
            __threadfence();
            s_ok = ok;
            if (!ok) atomicCAS(plan.err, 0, kErrBatchTimeout);
        }
        __syncthreads();
        if (!s_ok) return;
        const int steps = min(kB, J.T - b * kB);
        const uint32_t step0 = (uint32_t)(b * kB);
        const bool last = b == J.nblk - 1;
        const size_t plane = (size_t)J.H * J.P;
        if (J.form == 0) {  // discrete
            const uint8_t* in = (const uint8_t*)J.st[b & 1];
            bool burning = false;
#pragma unroll 4  // the loads of several iterations in flight together
            for (int i = tid; i < kRR * kRC; i += kBThreads) {
                const int y = i / kRC, x = i % kRC, gr = r0 + y, gc = c0 + x;
                const uint8_t v = (gr >= 0 && gr < J.H && gc >= 0 && gc < J.W) ? __ldcg(in + (size_t)gr * J.P + gc) : 0;
                s8[0][y][x] = v;
                s8[1][y][x] = v;
                burning |= v == 2;
            }
            // nothing burns in the region: no cell can change during the item's steps
            const int nsteps = __syncthreads_or(burning) ? steps : 0;
            if (tid == 0 && plan.stats) {
                const unsigned long long ic =
                    (unsigned long long)(min(kTR, J.H - ty * kTR) * min(kTC, J.W - tx * kTC)) * (unsigned long long)steps;
                atomicAdd(plan.stats + (nsteps ? kStatDisc : kStatDiscSkip), ic);
            }
            int cur = 0;
            for (int s = 0; s < nsteps; ++s) {
                for (int i = tid; i < (kRR - 2) * (kRC - 2); i += kBThreads) {
                    const int y = 1 + i / (kRC - 2), x = 1 + i % (kRC - 2), gr = r0 + y, gc = c0 + x;
                    const uint8_t sv = s8[cur][y][x];
                    uint8_t nv = sv;
                    if (sv == 1 || sv == 2) {  // states 1/2 exist only inside the grid
                        uint8_t nb[8];
#pragma unroll
                        for (int d = 0; d < 8; ++d) nb[d] = s8[cur][y + dir_dr(d)][x + dir_dc(d)];
                        nv = disc_update(sv, nb, J, J.q, plane, (size_t)gr * J.P + gc, (uint32_t)gr * (uint32_t)J.W + (uint32_t)gc,
                                         step0 + (uint32_t)s);
                    }
                    s8[cur ^ 1][y][x] = nv;
                }
                __syncthreads();
                cur ^= 1;
            }
            for (int i = tid; i < kTR * kTC; i += kBThreads) {
                const int y = kB + i / kTC, x = kB + i % kTC, gr = r0 + y, gc = c0 + x;
                if (gr >= J.H || gc >= J.W) continue;
                const uint8_t v = s8[cur][y][x];
                if (last) ((uint8_t*)J.out)[(size_t)gr * J.W + gc] = v;
                else ((uint8_t*)J.st[(b + 1) & 1])[(size_t)gr * J.P + gc] = v;
            }
        } else {
            // differentiable: A (decoded, own cell only) in sA[0], b and its tier in
            // ping-pong buffers (the tiers in the otherwise unused second half of sA)
            uint8_t(&sK)[2][kRR][kRC] = *reinterpret_cast<uint8_t(*)[2][kRR][kRC]>(&sA[1]);
            const float* in = (const float*)J.st[b & 1];
            bool burning = false;
#pragma unroll 4  // the loads of several iterations in flight together
            for (int i = tid; i < kRR * kRC; i += kBThreads) {
                const int y = i / kRC, x = i % kRC, gr = r0 + y, gc = c0 + x;
                const bool inside = gr >= 0 && gr < J.H && gc >= 0 && gc < J.W;
                const size_t g = (size_t)gr * J.P + gc;
                float Av = 0.0f, bv = 0.0f;
                int kv = 0;
                if (inside) x_decode(__ldcg(in + g), __ldcg(in + plane + g), Av, bv, kv);
                sA[0][y][x] = Av;
                sB[0][y][x] = bv;
                sB[1][y][x] = bv;
                sK[0][y][x] = (uint8_t)kv;
                sK[1][y][x] = (uint8_t)kv;
                burning |= bv != 0.0f;
            }
            // b = 0 in the whole region: every P is 0, the state does not change
            const bool live = __syncthreads_or(burning);
            if (tid == 0 && plan.stats) {
                const unsigned long long ic =
                    (unsigned long long)(min(kTR, J.H - ty * kTR) * min(kTC, J.W - tx * kTC)) * (unsigned long long)steps;
                atomicAdd(plan.stats + (live ? kStatDiff : kStatDiffSkip), ic);
            }
            int cur = 0;
            for (int s = 0; s < steps; ++s) {
                if (live) {
                    for (int i = tid; i < (kRR - 2) * (kRC - 2); i += kBThreads) {
                        const int y = 1 + i / (kRC - 2), x = 1 + i % (kRC - 2), gr = r0 + y, gc = c0 + x;
                        float bnew = sB[cur][y][x];
                        int knew = sK[cur][y][x];
                        if (gr >= 0 && gr < J.H && gc >= 0 && gc < J.W) {
                            const size_t qoff = (size_t)gr * J.P + gc;
                            float nb[8], qv[8];
                            int nk[8];
#pragma unroll
                            for (int d = 0; d < 8; ++d) {
                                nb[d] = sB[cur][y + dir_dr(d)][x + dir_dc(d)];
                                nk[d] = sK[cur][y + dir_dr(d)][x + dir_dc(d)];
                                qv[d] = __ldg(J.q + d * plane + qoff);
                            }
                            float An;
                            x_update(nb, nk, qv, sA[0][y][x], sB[cur][y][x], knew, J.pc, An, bnew, knew);
                            sA[0][y][x] = An;  // own cell only: in place
                        }
                        sB[cur ^ 1][y][x] = bnew;
                        sK[cur ^ 1][y][x] = (uint8_t)knew;
                    }
                    __syncthreads();
                    cur ^= 1;
                }
                if (J.tape) {  // the state at step0 + s + 1 of the interior, for the adjoint
                    float* o = J.tape + (size_t)(step0 + s + 1) * 2 * plane;
                    for (int i = tid; i < kTR * kTC; i += kBThreads) {
                        const int y = kB + i / kTC, x = kB + i % kTC, gr = r0 + y, gc = c0 + x;
                        if (gr >= J.H || gc >= J.W) continue;
                        x_encode(sA[0][y][x], sB[cur][y][x], sK[cur][y][x], o[(size_t)gr * J.P + gc],
                                 o[plane + (size_t)gr * J.P + gc]);
                    }
                }
            }
            for (int i = tid; i < kTR * kTC; i += kBThreads) {
                const int y = kB + i / kTC, x = kB + i % kTC, gr = r0 + y, gc = c0 + x;
                if (gr >= J.H || gc >= J.W) continue;
                const float Av = sA[0][y][x], bv = sB[cur][y][x];
                const int kv = sK[cur][y][x];
                if (last) {
                    // the output in plain FP32 (a tier's values read as 0 below FP32's range)
                    float* o = (float*)J.out;
                    o[(size_t)gr * J.W + gc] = signbit(Av) ? 1.0f + Av : Av * tier_scale(kv);
                    o[(size_t)J.H * J.W + (size_t)gr * J.W + gc] = bv * tier_scale(kv);
                } else {
                    float* o = (float*)J.st[(b + 1) & 1];
                    x_encode(Av, bv, kv, o[(size_t)gr * J.P + gc], o[plane + (size_t)gr * J.P + gc]);
                }
            }
        }
        __threadfence();
        __syncthreads();
        if (tid == 0 && !(plan.withhold && j == 0 && tile == 0 && J.nblk > 1 && b == 0)) {
            atomicExch(J.gen + tile, b + 1);
        }
    }
}

// ------------------------------------------------------------------ adjoint
// Work item (job, backward tile, rb): the adjoint of the job's block b = nblk - 1 - rb,
// steps t = t1 - 1 .. t0 (the same blocks as the forward), over a 16 x 32 interior with
// a 5-cell halo: per step the valid region shrinks by one cell, and the targets' own
// lambda at t + 1 must be valid one ring beyond the sources. lambda at t1 (scaled form,
// common.cuh) is read from the job's ping-pong buffer (b + 1) % 2 and lambda at t0 is
// written to b % 2; the item starts once the 3 x 3 neighbouring tiles have finished
// rb - 1 (so their lambda at t1 is there and they no longer read buffer b % 2).
// dL/dq of the interior is accumulated in the job's Gq (the tile's items run one after
// another, so the read-modify-write has no concurrent writer). Each step is the
// arithmetic of k_adjoint_step.
constexpr int kAR = 16, kAC = 32, kAH = kB + 1;
constexpr int kARR = kAR + 2 * kAH, kARC = kAC + 2 * kAH;  // 26 x 42
constexpr int kAThreads = 256;
constexpr int kTargets = (kARR - 2) * (kARC - 2);                 // targets of a step
constexpr int kTPT = (kTargets + kAThreads - 1) / kAThreads;       // targets per thread
constexpr int kSPT = (kARR * kARC + kAThreads - 1) / kAThreads;    // staged cells per thread

struct AdjSmem {
    float mua[kARR][kARC], mub[kARR][kARC];  // scaled lambda (mu) at t + 1, then at t
    float sa[kARR][kARC];                    // stored A at t
    float sb[kARR][kARC];                    // b at t in tier 0, 0 in the tiers (their 1 - b q is 1)
    float sbs[kARR][kARC];                   // b at t in its tier's units, b 2^(64 sigma)
    int ss[kARR][kARC];                      // sigma(t) (the tier)
    float sc[8][kARR][kARC];                 // contributions of targets, in source units
    float gq[8][kAR][kAC];                   // the item's dL/dq of the interior
    uint8_t sg[kARR][kARC];                  // sigma at t + 1, then at t
    int live;
};

__global__ void __launch_bounds__(kAThreads) k_batch_adj(BatchPlan plan) {
    extern __shared__ __align__(16) uint8_t adj_raw[];
    AdjSmem& sm = *reinterpret_cast<AdjSmem*>(adj_raw);
    __shared__ long long s_item;
    __shared__ int s_ok;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_item = (*(volatile int*)plan.err) ? plan.total : (long long)atomicAdd(plan.counter, 1ull);
        __syncthreads();
        const long long item = s_item;
        if (item >= plan.total) return;
        const int rb = upper_bound_ll(plan.blk_start, plan.max_blk + 1, item) - 1;
        const long long r = item - plan.blk_start[rb];
        const int j = upper_bound_ll(plan.tile_pref, plan.jobs_in_blk[rb] + 1, r) - 1;
        const int tile = (int)(r - plan.tile_pref[j]);
        const BatchJobDev& J = plan.jobs[j];
        const int ty = tile / J.btiles_x, tx = tile % J.btiles_x;
        const int r0 = ty * kAR - kAH, c0 = tx * kAC - kAH;
        if (tid == 0) {
            int ok = 1;
            for (int dy = -1; dy <= 1 && ok; ++dy)
                for (int dx = -1; dx <= 1 && ok; ++dx) {
                    const int yy = ty + dy, xx = tx + dx;
                    if (yy < 0 || yy >= J.btiles_y || xx < 0 || xx >= J.btiles_x) continue;
                    const volatile int* g = J.gen_b + yy * J.btiles_x + xx;
                    if (*g >= rb) continue;
                    const unsigned long long tw = global_ns();
                    while (*g < rb) {
                        if (global_ns() - tw > (unsigned long long)plan.wait_limit_ns || *(volatile int*)plan.err) {
                            ok = 0;
                            break;
                        }
                        __nanosleep(100);
                    }
                }
            __threadfence();
            s_ok = ok;
            if (!ok) atomicCAS(plan.err, 0, kErrBatchTimeout);
        }
        __syncthreads();
        if (!s_ok) return;
        const int b = J.nblk - 1 - rb;
        const int t0 = b * kB, t1 = min(J.T, t0 + kB);
        const size_t plane = (size_t)J.H * J.P;
        // a = 0 in the whole region at t1 - 1 (so at every step of the item, a never
        // decreases): every lambda ends masked to 0 and every dL/dq term has b_i = 0
        {
            bool any = t1 <= t0;  // no steps: lambda is carried over unchanged
            if (!any) {
                const float* st = J.tape + (size_t)(t1 - 1) * 2 * plane;
                for (int i = tid; i < kARR * kARC; i += kAThreads) {
                    const int y = i / kARC, x = i % kARC, gr = r0 + y, gc = c0 + x;
                    if (gr >= 0 && gr < J.H && gc >= 0 && gc < J.W)
                        any |= __float_as_uint(__ldcg(st + (size_t)gr * J.P + gc)) != 0u;
                }
            }
            const bool live_item = __syncthreads_or(any);
            if (tid == 0 && plan.stats) {
                const unsigned long long ic = (unsigned long long)(min(kAR, J.H - ty * kAR) * min(kAC, J.W - tx * kAC)) *
                                              (unsigned long long)max(0, t1 - t0);
                atomicAdd(plan.stats + (live_item ? kStatAdj : kStatAdjSkip), ic);
            }
            if (!live_item) {
                float* lo = J.lam[b & 1];
                uint8_t* so = J.sig[b & 1];
                for (int i = tid; i < kAR * kAC; i += kAThreads) {
                    const int gr = r0 + kAH + i / kAC, gc = c0 + kAH + i % kAC;
                    if (gr >= J.H || gc >= J.W) continue;
                    const size_t g = (size_t)gr * J.P + gc;
                    lo[g] = 0.0f;
                    lo[plane + g] = 0.0f;
                    so[g] = (uint8_t)kSigmaZero;
                }
                __threadfence();
                __syncthreads();
                if (tid == 0) atomicExch(J.gen_b + tile, rb + 1);
                continue;
            }
        }
        for (int i = tid; i < 8 * kAR * kAC; i += kAThreads) (&sm.gq[0][0][0])[i] = 0.0f;
        // lambda at t1 over the whole region
        {
            const float* lin = J.lam[(b + 1) & 1];
            const uint8_t* sin_ = J.sig[(b + 1) & 1];
            for (int i = tid; i < kARR * kARC; i += kAThreads) {
                const int y = i / kARC, x = i % kARC, gr = r0 + y, gc = c0 + x;
                const bool in = gr >= 0 && gr < J.H && gc >= 0 && gc < J.W;
                const size_t g = (size_t)gr * J.P + gc;
                sm.mua[y][x] = in ? __ldcg(lin + g) : 0.0f;
                sm.mub[y][x] = in ? __ldcg(lin + plane + g) : 0.0f;
                sm.sg[y][x] = in ? __ldcg(sin_ + g) : (uint8_t)kSigmaZero;
            }
        }
        // q of this thread's targets (at most kTPT of them), read once for the item's steps
        float qt[kTPT][8];
#pragma unroll
        for (int u = 0; u < kTPT; ++u) {
            const int i = tid + u * kAThreads;
            const int y = 1 + i / (kARC - 2), x = 1 + i % (kARC - 2), gr = r0 + y, gc = c0 + x;
            const bool ok = i < kTargets && gr >= 0 && gr < J.H && gc >= 0 && gc < J.W;
            const size_t g = ok ? (size_t)gr * J.P + gc : 0;
#pragma unroll
            for (int d = 0; d < 8; ++d) qt[u][d] = ok ? __ldg(J.q + d * plane + g) : 0.0f;
        }
        for (int t = t1 - 1; t >= t0; --t) {
            const float* st = J.tape + (size_t)t * 2 * plane;
            // the region's state at t (every load of the thread issued before any store)
            float As_[kSPT], Bs_[kSPT];
#pragma unroll
            for (int u = 0; u < kSPT; ++u) {
                const int i = tid + u * kAThreads;
                const int y = i / kARC, x = i % kARC, gr = r0 + y, gc = c0 + x;
                const bool in = i < kARR * kARC && gr >= 0 && gr < J.H && gc >= 0 && gc < J.W;
                const size_t g = in ? (size_t)gr * J.P + gc : 0;
                As_[u] = in ? __ldcg(st + g) : 0.0f;
                Bs_[u] = in ? __ldcg(st + plane + g) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < kSPT; ++u) {
                const int i = tid + u * kAThreads;
                if (i >= kARR * kARC) continue;
                const int y = i / kARC, x = i % kARC, gr = r0 + y, gc = c0 + x;
                const bool in = gr >= 0 && gr < J.H && gc >= 0 && gc < J.W;
                const float As = As_[u], Bs = Bs_[u];
                sm.sa[y][x] = As;
                sm.sb[y][x] = fmaxf(Bs, 0.0f);
                sm.sbs[y][x] = fabsf(Bs);
                sm.ss[y][x] = in ? x_sigma(As, Bs) : kSigmaZero;
            }
            __syncthreads();
            // targets j: contributions to their sources and, in the interior, dL/dq
#pragma unroll
            for (int u = 0; u < kTPT; ++u) {
                const int i = tid + u * kAThreads;
                if (i >= kTargets) continue;
                const int y = 1 + i / (kARC - 2), x = 1 + i % (kARC - 2), gr = r0 + y, gc = c0 + x;
                const int sgp = sm.sg[y][x];
                if (sgp == kSigmaZero || gr < 0 || gr >= J.H || gc < 0 || gc >= J.W) {
#pragma unroll
                    for (int d = 0; d < 8; ++d) sm.sc[d][y][x] = 0.0f;
                    continue;
                }
                float qd[8], f[8];
#pragma unroll
                for (int d = 0; d < 8; ++d) {
                    qd[d] = qt[u][d];
                    f[d] = fmaf(-sm.sb[y + dir_dr(d)][x + dir_dc(d)], qd[d], 1.0f);
                }
                float pre[8], suf[8];
                pre[0] = 1.0f;
#pragma unroll
                for (int d = 1; d < 8; ++d) pre[d] = pre[d - 1] * f[d - 1];
                suf[7] = 1.0f;
#pragma unroll
                for (int d = 6; d >= 0; --d) suf[d] = suf[d + 1] * f[d + 1];
                const float P = 1.0f - pre[7] * f[7];
                const float la = sm.mua[y][x], lb = sm.mub[y][x];
                const float ln = la + lb;
                const float As = sm.sa[y][x];
                const int sj = sm.ss[y][x];
                // 1 - a (1 in the tiers below 2^-64)
                const float ua = signbit(As) ? -As : (sj >= 1 && sj != kSigmaZero ? 1.0f : 1.0f - As);
                const float tg = ln * ua;
                const bool interior = y >= kAH && y < kAH + kAR && x >= kAH && x < kAH + kAC;
#pragma unroll
                for (int d = 0; d < 8; ++d) {
                    const int yy = y + dir_dr(d), xx = x + dir_dc(d);
                    const float tt = tg * (pre[d] * suf[d]);
                    const float r_d = exp2i(64 * (sgp - sm.ss[yy][xx]));
                    sm.sc[d][y][x] = tt * qd[d] * r_d;
                    if (interior)
                        sm.gq[d][y - kAH][x - kAH] = fmaf(tt, sm.sbs[yy][xx] * r_d, sm.gq[d][y - kAH][x - kAH]);
                }
                sm.mua[y][x] = fmaf(-ln, P, la) * exp2i(64 * (sgp - sj));  // own cell: in place
            }
            __syncthreads();
            // sources i: lambda_b at t, and the masks of cells with a = 0
            for (int i = tid; i < (kARR - 4) * (kARC - 4); i += kAThreads) {
                const int y = 2 + i / (kARC - 4), x = 2 + i % (kARC - 4), gr = r0 + y, gc = c0 + x;
                const bool in = gr >= 0 && gr < J.H && gc >= 0 && gc < J.W;
                const int sgp = sm.sg[y][x];
                const int sgt = in ? sm.ss[y][x] : kSigmaZero;
                float acc = 0.0f;
                if (sgp != kSigmaZero) acc = J.pc * sm.mub[y][x] * exp2i(64 * (sgp - sgt));
#pragma unroll
                for (int d = 0; d < 8; ++d) acc += sm.sc[d][y - dir_dr(d)][x - dir_dc(d)];
                if (sgt == kSigmaZero || sgp == kSigmaZero) {
                    acc = 0.0f;
                    sm.mua[y][x] = 0.0f;
                }
                sm.mub[y][x] = acc;
                sm.sg[y][x] = (uint8_t)sgt;
            }
            __syncthreads();
        }
        // lambda at t0 and the item's dL/dq of the interior (one read-modify-write per item)
        {
            float* lo = J.lam[b & 1];
            uint8_t* so = J.sig[b & 1];
            for (int i = tid; i < kAR * kAC; i += kAThreads) {
                const int y = kAH + i / kAC, x = kAH + i % kAC, gr = r0 + y, gc = c0 + x;
                if (gr >= J.H || gc >= J.W) continue;
                const size_t g = (size_t)gr * J.P + gc;
                lo[g] = sm.mua[y][x];
                lo[plane + g] = sm.mub[y][x];
                so[g] = sm.sg[y][x];
#pragma unroll
                for (int d = 0; d < 8; ++d) J.Gq[d * plane + g] += sm.gq[d][i / kAC][i % kAC];
            }
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) atomicExch(J.gen_b + tile, rb + 1);
    }
}

}  // namespace

int batch_tile_rows() { return kTR; }
int batch_tile_cols() { return kTC; }
int batch_steps_per_item() { return kB; }

void launch_batch(const BatchPlan& plan, int grid, cudaStream_t s) {
    k_batch<<<grid, kBThreads, 0, s>>>(plan);
}

int batch_adj_tile_rows() { return kAR; }
int batch_adj_tile_cols() { return kAC; }

int batch_adj_configure() {
    static int done = 0;
    if (!done) {
        if (cudaFuncSetAttribute(k_batch_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(AdjSmem)) !=
            cudaSuccess)
            return -1;
        done = 1;
    }
    return 0;
}

int batch_adj_blocks_per_sm() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_adj, kAThreads, sizeof(AdjSmem)) != cudaSuccess)
        nb = 1;
    return nb > 0 ? nb : 1;
}

void launch_batch_adj(const BatchPlan& plan, int grid, cudaStream_t s) {
    k_batch_adj<<<grid, kAThreads, sizeof(AdjSmem), s>>>(plan);
}

int batch_blocks_per_sm() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch, kBThreads, 0) != cudaSuccess) nb = 1;
    return nb > 0 ? nb : 1;
}

}  // namespace pf
