// Discrete stochastic step (Sec. 2.2 transition rules, Eq. 9): uint8 states packed
// four per 32-bit word, SWAR "any neighbour burning" tests, Philox draws taken only
// for cells that can change.
//   - k_discrete_step: the plain one-launch-per-step kernel (global memory only).
//   - k_discrete_blocked: TMA-staged tile + halo, k steps per launch in shared memory.
#include <cuda.h>

#include "common.cuh"
#include "tma.cuh"
#include "prep_math.cuh"

namespace pf {

namespace {

// Burning flags (bit 0 of each byte) of cells c-1 .. c+4 of one row, as bytes 0..5 of
// a 64-bit word, from the word at c..c+3 and its left / right neighbour words.
__device__ __forceinline__ uint64_t row_burning(uint32_t left, uint32_t mid, uint32_t right) {
    const uint64_t ext = (uint64_t)(left >> 24) | ((uint64_t)mid << 8) | ((uint64_t)(right & 0xffu) << 40);
    return (ext >> 1) & ~ext & 0x0101010101010101ull;
}

// New value of the 4 cells of word `mid` (row r, columns col0..col0+3 of the grid).
// U/C/D are the burning flags of the rows above / at / below (row_burning layout).
// ties: near-tie counts of this call's owned cells (ignition in the low 16 bits,
// continue in the high 16 bits), added to.
// kLoop: the draws of the word's cells in one loop over its drawing cells, so that every
// lane of a warp with a draw left runs the same Philox code together, whichever of its 4
// cells it is for (faster in the plain kernel); else a branch per cell (faster in the
// blocked kernel, whose words are denser in drawing cells). The same arithmetic either way.
template <bool kLoop>
__device__ __forceinline__ uint32_t update_word(uint32_t mid, uint64_t U, uint64_t C, uint64_t D, int r,
                                                int col0, size_t qoff, size_t qplane, const float* __restrict__ q,
                                                const DiscreteArgs& g, uint32_t run, uint32_t step, int rr,
                                                uint32_t& ties, const PrepArgs* pa = nullptr) {
    const uint64_t all3 = U | C | D;
    const uint64_t nb64 = (all3 << 8) | (all3 >> 8) | U | D;  // neighbours of byte positions 1..4
    const uint32_t nb = (uint32_t)(nb64 >> 8) & 0x01010101u;
    const uint32_t burning = lanes_eq2(mid);
    const uint32_t active = burning | (nb & lanes_eq1(mid));
    if (active == 0u) return mid;
    // the probability a drawing cell's uniform is compared with: Eq. 9 over the burning
    // neighbours for an unburned cell, as P <- P + x (1 - P), with q read from the
    // materialised planes or (pa) recomputed from the fields with prep's arithmetic;
    // p_continue for a burning one
    auto threshold = [&](int k) {
        float qv[8];
        if (pa) q_cell(*pa, r, col0 + k, qv);
        float P = 0.0f;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const uint64_t row = dir_dr(d) < 0 ? U : (dir_dr(d) == 0 ? C : D);
            if ((row >> (8 * (k + 1 + dir_dc(d)))) & 1ull) {
                const float x = pa ? qv[d] : __ldg(q + (size_t)d * qplane + qoff + k);
                P = fmaf(x, 1.0f - P, P);
            }
        }
        return P;
    };
    // the draw of cell k against t: its new state, the accumulator and the near-ties
    auto draw = [&](int k, bool unburned, float t) {
        const int col = col0 + k;
        const uint32_t cell = (uint32_t)r * (uint32_t)g.W + (uint32_t)col;
        const U4 x = philox10(cell, run, step, g.fire, g.key0, g.key1);
        const float u = u24(unburned ? x.x : x.y);
        const uint32_t ns = (u < t) ? 2u : (unburned ? 1u : 3u);
        const bool owned = r >= g.acc_r0 && r < g.acc_r1 && col >= g.acc_c0 && col < g.acc_c1;
        if (unburned && ns == 2u && g.acc && owned)
            g.acc[((size_t)rr * g.H + r) * g.W + col] = t;  // the accumulator (Sec. 2.2 data flow)
        ties += (owned && fabsf(u - t) < kNearTie) ? (unburned ? 1u : 0x10000u) : 0u;
        return ns;
    };
    uint32_t out = mid;
    if constexpr (kLoop) {
        float thr[4];
        uint32_t ign = 0u;  // bytes of the unburned drawing cells
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            thr[k] = g.p_continue;
            if (((active >> (8 * k)) & 1u) == 0u || ((mid >> (8 * k)) & 0xffu) != 1u) continue;
            ign |= 1u << (8 * k);
            thr[k] = threshold(k);
        }
        for (uint32_t pend = active; pend != 0u; pend &= pend - 1u) {
            const int k = (__ffs((int)pend) - 1) >> 3;
            const float t = k == 0 ? thr[0] : (k == 1 ? thr[1] : (k == 2 ? thr[2] : thr[3]));
            const uint32_t ns = draw(k, (ign >> (8 * k)) & 1u, t);
            out = (out & ~(0xffu << (8 * k))) | (ns << (8 * k));
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (((active >> (8 * k)) & 1u) == 0u) continue;
            const bool unburned = ((mid >> (8 * k)) & 0xffu) == 1u;
            const uint32_t ns = draw(k, unburned, unburned ? threshold(k) : g.p_continue);
            out = (out & ~(0xffu << (8 * k))) | (ns << (8 * k));
        }
    }
    return out;
}

// Adds a thread's near-tie counts to the global counters: one reduction per warp, and
// atomics only from warps that saw a tie (they are rare). Every lane of the warp calls this.
__device__ __forceinline__ void flush_ties(const DiscreteArgs& g, uint32_t ties) {
    if (!g.ties || !__any_sync(0xffffffffu, ties != 0u)) return;
    const uint32_t ign = __reduce_add_sync(0xffffffffu, ties & 0xffffu);
    const uint32_t con = __reduce_add_sync(0xffffffffu, ties >> 16);
    if ((threadIdx.x & 31) == 0) {
        if (ign) atomicAdd(g.ties, (unsigned long long)ign);
        if (con) atomicAdd(g.ties + 1, (unsigned long long)con);
    }
}

// rc: q recomputed from the fields (prep's arithmetic) instead of read from q
template <bool rc>
__global__ void __launch_bounds__(256) k_discrete_step(DiscreteArgs g, const uint8_t* __restrict__ S,
                                                       uint8_t* __restrict__ Sn, const float* __restrict__ q,
                                                       uint32_t step, const __grid_constant__ PrepArgs pa) {
    const int wpr = g.pitch >> 2;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)g.R * g.H * wpr;
    uint32_t ties = 0u;
    if (idx < total) {
        const int w = (int)(idx % wpr);
        const size_t rowid = idx / wpr;
        const int r = (int)(rowid % g.H);
        const int rr = (int)(rowid / g.H);
        const uint32_t* base = reinterpret_cast<const uint32_t*>(S + (size_t)rr * g.H * g.pitch);
        auto ld = [&](int y, int x) -> uint32_t {
            return (y >= 0 && y < g.H && x >= 0 && x < wpr) ? __ldg(base + (size_t)y * wpr + x) : 0u;
        };
        const uint32_t mid = ld(r, w);
        const uint64_t U = row_burning(ld(r - 1, w - 1), ld(r - 1, w), ld(r - 1, w + 1));
        const uint64_t C = row_burning(ld(r, w - 1), mid, ld(r, w + 1));
        const uint64_t D = row_burning(ld(r + 1, w - 1), ld(r + 1, w), ld(r + 1, w + 1));
        const uint32_t out = update_word<true>(mid, U, C, D, r, 4 * w, (size_t)r * g.pitch + 4 * w,
                                         (size_t)g.H * g.pitch, q, g, g.run0 + (uint32_t)rr, step, rr, ties,
                                         rc ? &pa : nullptr);
        reinterpret_cast<uint32_t*>(Sn + (size_t)rr * g.H * g.pitch)[(size_t)r * wpr + w] = out;
    }
    flush_ties(g, ties);  // every lane of the warp, converged
}

// ------------------------------------------------------------ temporal-blocked
// Tile: kTW interior bytes x TH interior rows; the TMA box adds 16 bytes left and right
// (TMA x offsets must be 16-byte multiples, so k <= 16) and k rows above and below.
constexpr int kTW = 128;
constexpr int kXH = 16;
constexpr int kCT = kTW + 2 * kXH;  // 160 bytes per tile row
constexpr int kCW = kCT / 4;        // 40 words per tile row
constexpr int kBlkThreads = 256;

// kRc: q recomputed from the fields of pa (prep's arithmetic) instead of read from q
template <bool kRc>
__global__ void __launch_bounds__(kBlkThreads) k_discrete_blocked(const __grid_constant__ CUtensorMap tin,
                                                                  const __grid_constant__ PrepArgs pa,
                                                                  DiscreteArgs g, int TH, int KH,
                                                                  uint8_t* __restrict__ Sn,
                                                                  const float* __restrict__ q, uint32_t step0,
                                                                  int k, int* __restrict__ err, TmaHook hk,
                                                                  unsigned long long* __restrict__ skipped) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    // TMA destinations: round the dynamic shared-memory base up to 128 bytes (the
    // allocation carries 128 bytes of slack for this)
    uint8_t* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    __shared__ int any_burning;
    const int RT = TH + 2 * KH;
    const int tile_bytes = RT * kCT;
    uint32_t* A = reinterpret_cast<uint32_t*>(smem);
    uint32_t* B = reinterpret_cast<uint32_t*>(smem + ((tile_bytes + 127) & ~127));
    const int c0 = blockIdx.x * kTW;
    const int r0 = blockIdx.y * TH;
    const int rr = blockIdx.z;
    if (threadIdx.x == 0) {
        any_burning = 0;
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, (uint32_t)tile_bytes);
        if (!hk.withhold) tma_load_3d(A, &tin, &bar, c0 - kXH, r0 - KH, rr);
    }
    const bool ok = mbar_wait_bounded(&bar, 0, hk.spin);
    if (!__syncthreads_and(ok)) {
        if (threadIdx.x == 0) {
            atomicExch(err, kErrTmaTimeout);
            mbar_wait_bounded(&bar, 0, hk.spin);  // give the copy in flight one more budget
        }
        return;
    }
    // Copy A -> B so the ring the steps never write holds defined states, and find
    // whether anything burns in the tile at all.
    const int nwords = tile_bytes / 4;
    int local_burn = 0;
    for (int i = threadIdx.x; i < nwords; i += kBlkThreads) {
        const uint32_t v = A[i];
        B[i] = v;
        local_burn |= (lanes_eq2(v) != 0u);
    }
    if (local_burn) any_burning = 1;
    __syncthreads();
    const size_t qplane = (size_t)g.H * g.pitch;
    uint32_t* src = A;
    uint32_t* dst = B;
    // the accumulator is written by the tile that owns a cell's interior position
    DiscreteArgs ga = g;
    ga.acc_r0 = r0;
    ga.acc_r1 = r0 + TH;
    ga.acc_c0 = c0;
    ga.acc_c1 = c0 + kTW < g.W ? c0 + kTW : g.W;
    uint32_t ties = 0u;
    // nothing burns in the tile: no cell can change during the launch (its steps are
    // skipped; the interior is still stored)
    if (!any_burning && skipped && threadIdx.x == 0) {
        const int rows = min(TH, g.H - r0), cols = min(kTW, g.W - c0);
        if (rows > 0 && cols > 0) atomicAdd(skipped, (unsigned long long)rows * cols * k);
    }
    if (any_burning) {
        const int y_off = r0 - KH, x_off = c0 - kXH;
        for (int s = 0; s < k; ++s) {
            // rows / words that can still influence the interior after step s
            const int y_lo = KH - k + 1 + s, y_hi = RT - y_lo;  // rows [y_lo, y_hi)
            const int b_lo = kXH - k + 1 + s;                                   // first byte needed
            int m_lo = b_lo >> 2, m_hi = (kCT - 1 - b_lo) >> 2;
            m_lo = m_lo < 1 ? 1 : m_lo;
            m_hi = m_hi > kCW - 2 ? kCW - 2 : m_hi;
            const int nm = m_hi - m_lo + 1, ny = y_hi - y_lo;
            const uint32_t step = step0 + (uint32_t)s;
            for (int i = threadIdx.x; i < nm * ny; i += kBlkThreads) {
                const int y = y_lo + i / nm, m = m_lo + i % nm;
                const uint32_t* ru = src + (y - 1) * kCW;
                const uint32_t* rc = src + y * kCW;
                const uint32_t* rd = src + (y + 1) * kCW;
                const uint32_t mid = rc[m];
                const uint64_t U = row_burning(ru[m - 1], ru[m], ru[m + 1]);
                const uint64_t C = row_burning(rc[m - 1], mid, rc[m + 1]);
                const uint64_t D = row_burning(rd[m - 1], rd[m], rd[m + 1]);
                const int gr = y_off + y, gc = x_off + 4 * m;
                // states 1/2 exist only inside the grid, so gr/gc are valid whenever a
                // cell is active; the q offset is formed but only read for such cells
                const size_t qoff = (size_t)gr * g.pitch + gc;
                dst[y * kCW + m] = update_word<false>(mid, U, C, D, gr, gc, qoff, qplane, q, ga, g.run0 + (uint32_t)rr, step,
                                               rr, ties, kRc ? &pa : nullptr);
            }
            __syncthreads();
            uint32_t* t = src; src = dst; dst = t;
        }
    }
    flush_ties(g, ties);
    // store the interior rows [KH, KH + TH), bytes [16, 144) with 16-byte vectors
    uint8_t* out = Sn + (size_t)rr * g.H * g.pitch;
    const int vec_per_row = kTW / 16;
    for (int i = threadIdx.x; i < TH * vec_per_row; i += kBlkThreads) {
        const int y = i / vec_per_row, v = i % vec_per_row;
        const int gr = r0 + y, gc = c0 + 16 * v;
        if (gr >= g.H || gc >= g.pitch) continue;
        const uint4 val = *reinterpret_cast<const uint4*>(reinterpret_cast<const uint8_t*>(src) + (KH + y) * kCT + kXH + 16 * v);
        *reinterpret_cast<uint4*>(out + (size_t)gr * g.pitch + gc) = val;
    }
}

// DCA gradient of one step: thread per cell, realisations summed in order (no atomics).
__global__ void __launch_bounds__(256) k_dca_step(DiscreteArgs g, const uint8_t* __restrict__ S,
                                                  const uint8_t* __restrict__ Sn, const float* __restrict__ q,
                                                  const float* __restrict__ w, float* __restrict__ Gq) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t HW = (size_t)g.H * g.W;
    if (idx >= HW) return;
    const int r = (int)(idx / g.W), c = (int)(idx % g.W);
    const size_t plane = (size_t)g.H * g.pitch;
    const size_t j = (size_t)r * g.pitch + c;
    float G[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    bool any = false;
    for (int rr = 0; rr < g.R; ++rr) {
        const size_t o = (size_t)rr * plane;
        if (S[o + j] != 1 || Sn[o + j] != 2) continue;
        const float wj = __ldg(w + (size_t)rr * HW + idx);
        if (wj == 0.0f) continue;
        any = true;
        float beta[8], f[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const int ri = r + dir_dr(d), ci = c + dir_dc(d);
            beta[d] = (ri >= 0 && ri < g.H && ci >= 0 && ci < g.W && S[o + (size_t)ri * g.pitch + ci] == 2) ? 1.0f : 0.0f;
            f[d] = fmaf(-beta[d], __ldg(q + d * plane + j), 1.0f);
        }
        // leave-one-out products by prefix / suffix (no division: a factor can be 0)
        float pre[8], suf[8];
        pre[0] = 1.0f;
#pragma unroll
        for (int d = 1; d < 8; ++d) pre[d] = pre[d - 1] * f[d - 1];
        suf[7] = 1.0f;
#pragma unroll
        for (int d = 6; d >= 0; --d) suf[d] = suf[d + 1] * f[d + 1];
#pragma unroll
        for (int d = 0; d < 8; ++d) G[d] = fmaf(wj * beta[d], pre[d] * suf[d], G[d]);
    }
    if (!any) return;
#pragma unroll
    for (int d = 0; d < 8; ++d) Gq[d * plane + j] += G[d];
}

__global__ void k_ignition_map_discrete(DiscreteArgs g, const uint8_t* __restrict__ S, const float* __restrict__ q,
                                        float* __restrict__ P) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t HW = (size_t)g.H * g.W;
    if (idx >= HW * g.R) return;
    const int rr = (int)(idx / HW);
    const size_t j = idx % HW;
    const int r = (int)(j / g.W), c = (int)(j % g.W);
    const uint8_t* s = S + (size_t)rr * g.H * g.pitch;
    float p = 0.0f;
    if (s[(size_t)r * g.pitch + c] == 1) {
        for (int d = 0; d < 8; ++d) {
            const int ri = r + dir_dr(d), ci = c + dir_dc(d);
            if (ri < 0 || ri >= g.H || ci < 0 || ci >= g.W) continue;
            if (s[(size_t)ri * g.pitch + ci] == 2) {
                const float x = q[(size_t)d * g.H * g.pitch + (size_t)r * g.pitch + c];
                p = fmaf(x, 1.0f - p, p);
            }
        }
    }
    P[idx] = p;
}

}  // namespace

void launch_discrete_step(const DiscreteArgs& g, const uint8_t* S, uint8_t* Sn, const float* q, uint32_t step,
                          cudaStream_t s) {
    const size_t total = (size_t)g.R * g.H * (g.pitch >> 2);
    const unsigned blocks = (unsigned)((total + 255) / 256);
    k_discrete_step<false><<<blocks, 256, 0, s>>>(g, S, Sn, q, step, PrepArgs{});
}

void launch_discrete_step_rc(const DiscreteArgs& g, const uint8_t* S, uint8_t* Sn, const PrepArgs& pa, uint32_t step,
                             cudaStream_t s) {
    const size_t total = (size_t)g.R * g.H * (g.pitch >> 2);
    const unsigned blocks = (unsigned)((total + 255) / 256);
    k_discrete_step<true><<<blocks, 256, 0, s>>>(g, S, Sn, nullptr, step, pa);
}

void launch_dca_step(const DiscreteArgs& g, const uint8_t* S, const uint8_t* Sn, const float* q, const float* w,
                     float* Gq, cudaStream_t s) {
    const size_t HW = (size_t)g.H * g.W;
    k_dca_step<<<(unsigned)((HW + 255) / 256), 256, 0, s>>>(g, S, Sn, q, w, Gq);
}

int discrete_blocked_tile_rows() { return 64; }
// The first and last 4-byte words of a staged row are never updated (their outer
// neighbour word is not staged), so the kXH-byte column halo supports kXH - 3 steps per
// launch; a multiple of 4 below that.
int discrete_blocked_max_k() { return kXH - 4; }

size_t discrete_blocked_smem(int TH, int KH) {
    const int tile_bytes = (TH + 2 * KH) * kCT;
    return 2 * (size_t)((tile_bytes + 127) & ~127) + 128;
}

void launch_discrete_blocked_impl(const DiscreteArgs& g, const CUtensorMap* tin, int TH, int KH, uint8_t* Sn,
                                  const float* q, const PrepArgs* pa, uint32_t step, int k, int* err, TmaHook hk,
                                  unsigned long long* skipped, cudaStream_t s) {
    const size_t smem = discrete_blocked_smem(TH, KH);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_discrete_blocked<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        cudaFuncSetAttribute(k_discrete_blocked<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        attr_set = true;
    }
    dim3 grd((g.pitch + kTW - 1) / kTW, (g.H + TH - 1) / TH, g.R);
    if (pa)
        k_discrete_blocked<true><<<grd, kBlkThreads, smem, s>>>(*tin, *pa, g, TH, KH, Sn, nullptr, step, k, err, hk,
                                                                skipped);
    else
        k_discrete_blocked<false><<<grd, kBlkThreads, smem, s>>>(*tin, PrepArgs{}, g, TH, KH, Sn, q, step, k, err, hk,
                                                                 skipped);
}

void launch_ignition_map_discrete(const DiscreteArgs& g, const uint8_t* S, const float* q, float* P,
                                  cudaStream_t s) {
    const size_t total = (size_t)g.R * g.H * g.W;
    k_ignition_map_discrete<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(g, S, q, P);
}

}  // namespace pf
