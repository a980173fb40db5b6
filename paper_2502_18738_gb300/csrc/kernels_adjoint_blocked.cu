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
//   * writes lambda at t0 for the interior and adds the tile's dL/dq into global memory.
// The halo shrinks by one cell per step, so the 48 x 48 interior is exact for n <= 7.
#include <cuda.h>

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
};

__device__ __forceinline__ void origin(int tile, int tiles_x, int& r0, int& c0) {
    r0 = (tile / tiles_x) * kIR - kHalo;
    c0 = (tile % tiles_x) * kIC - kHalo;
}

__global__ void __launch_bounds__(kThreads, 1)
    k_adjoint_blocked(const __grid_constant__ CUtensorMap tst, const __grid_constant__ CUtensorMap tq, int H,
                      int pitch, float pc, int zlast, int n, int tiles_x, int ntiles,
                      const float* __restrict__ lam_in, float* __restrict__ lam_out, float* __restrict__ Gq,
                      int* __restrict__ err) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    __shared__ __align__(8) uint64_t sbar[2];
    __shared__ __align__(8) uint64_t qbar;
    __shared__ uint32_t tslot;

    const int tid = threadIdx.x;
    const int x = tid % kCT;
    const int strip = tid / kCT;
    const int ys = strip * kM;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const size_t gplane = (size_t)H * pitch;
    const int nloc = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    if (nloc <= 0) return;
    const int total = nloc * n;

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

    auto issue_state = [&](int i) {
        const int l = i / n, m = i % n;
        int r0, c0;
        origin((int)blockIdx.x + l * (int)gridDim.x, tiles_x, r0, c0);
        const int s = i & 1;
        mbar_arrive_expect_tx(&sbar[s], (uint32_t)(2 * kPlane * sizeof(float)));
        tma_load_3d(sm.st[s], &tst, &sbar[s], c0, r0, 2 * (zlast - m));
    };
    auto issue_q = [&](int l) {
        int r0, c0;
        origin((int)blockIdx.x + l * (int)gridDim.x, tiles_x, r0, c0);
        mbar_arrive_expect_tx(&qbar, (uint32_t)(8 * kPlane * sizeof(float)));
        tma_load_3d(sm.q, &tq, &qbar, c0, r0, 0);
    };
    if (tid == 0) {
        issue_q(0);
        issue_state(0);
        if (total > 1) issue_state(1);
    }

    bool failed = false;
    float la[kM], lb[kM];
    for (int l = 0; l < nloc && !failed; ++l) {
        const int tile = (int)blockIdx.x + l * (int)gridDim.x;
        int r0, c0;
        origin(tile, tiles_x, r0, c0);
        if (!__syncthreads_and(mbar_wait_bounded(&qbar, (uint32_t)(l & 1)))) {
            failed = true;
            break;
        }
        // prologue: q -> TMEM, dL/dq accumulator := 0, lambda' of the region -> registers
#pragma unroll
        for (int k = 0; k < kM; ++k) {
            const int y = ys + k;
            float qv[8], z[8];
#pragma unroll
            for (int d = 0; d < 8; ++d) {
                qv[d] = sm.q[d * kPlane + y * kCT + x];
                z[d] = 0.0f;
            }
            tmem_st8(tbase + 16 * k, qv);
            tmem_st8(tbase + 16 * k + 8, z);
            const int gr = r0 + y, gc = c0 + x;
            const bool in = gr >= 0 && gr < H && gc >= 0 && gc < pitch;
            la[k] = in ? lam_in[(size_t)gr * pitch + gc] : 0.0f;
            lb[k] = in ? lam_in[gplane + (size_t)gr * pitch + gc] : 0.0f;
        }
        tmem_wait_st();
        fence_proxy_async();
        __syncthreads();  // q stage consumed
        if (tid == 0 && l + 1 < nloc) issue_q(l + 1);

        for (int m = 0; m < n; ++m) {
            const int i = l * n + m;
            const int s = i & 1, ex = i & 1;
            if (!__syncthreads_and(mbar_wait_bounded(&sbar[s], (uint32_t)((i >> 1) & 1)))) {
                failed = true;
                break;
            }
            const float* stA = sm.st[s];
            const float* stB = sm.st[s] + kPlane;
            float acc[3][kM + 2];
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < kM + 2; ++k) acc[j][k] = 0.0f;
            const bool xin = x >= 1 && x < kCT - 1;
            const int xl = xin ? x - 1 : x, xr = xin ? x + 1 : x;
#pragma unroll
            for (int k = 0; k < kM; ++k) {
                const int y = ys + k;
                float qv[8], gv[8];
                tmem_ld8(tbase + 16 * k, qv);
                tmem_ld8(tbase + 16 * k + 8, gv);
                const int yu = y > 0 ? y - 1 : y, yd = y < kRT - 1 ? y + 1 : y;
                if (xin && y >= 1 && y < kRT - 1) {
                    // neighbours in direction order (-1,-1) (-1,0) (-1,1) (0,-1) (0,1) (1,-1) (1,0) (1,1)
                    const float nb[8] = {stB[yu * kCT + xl], stB[yu * kCT + x], stB[yu * kCT + xr],
                                         stB[y * kCT + xl],  stB[y * kCT + xr], stB[yd * kCT + xl],
                                         stB[yd * kCT + x],  stB[yd * kCT + xr]};
                    float f[8], P = 0.0f;
#pragma unroll
                    for (int d = 0; d < 8; ++d) {
                        const float xx = nb[d] * qv[d];
                        f[d] = 1.0f - xx;
                        P = fmaf(xx, 1.0f - P, P);
                    }
                    float pre[8], suf[8];
                    pre[0] = 1.0f;
#pragma unroll
                    for (int d = 1; d < 8; ++d) pre[d] = pre[d - 1] * f[d - 1];
                    suf[7] = 1.0f;
#pragma unroll
                    for (int d = 6; d >= 0; --d) suf[d] = suf[d + 1] * f[d + 1];
                    float av, ua;
                    a_decode(stA[y * kCT + x], av, ua);
                    const float ln = la[k] + lb[k];
                    const float lP = ln * ua;
                    la[k] = la[k] - ln * P;
#pragma unroll
                    for (int d = 0; d < 8; ++d) {
                        const float loo = pre[d] * suf[d];
                        gv[d] = fmaf(lP * nb[d], loo, gv[d]);
                        acc[dir_dc(d) + 1][k + 1 + dir_dr(d)] += lP * qv[d] * loo;
                    }
                }
                tmem_st8(tbase + 16 * k + 8, gv);
            }
            tmem_wait_st();
            // publish the contributions that leave this thread's strip or warp
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                sm.vtop[ex][strip][j][x] = acc[j][0];
                sm.vbot[ex][strip][j][x] = acc[j][kM + 1];
            }
            if (x == 31) {
#pragma unroll
                for (int k = 0; k < kM; ++k) sm.el2r[ex][strip][k] = acc[2][k + 1];
            }
            if (x == 32) {
#pragma unroll
                for (int k = 0; k < kM; ++k) sm.er2l[ex][strip][k] = acc[0][k + 1];
            }
            fence_proxy_async();  // stage s fully read before it is refilled by TMA
            __syncthreads();
            if (tid == 0 && i + 2 < total) issue_state(i + 2);
            // gather: lambda_b at the sources of this strip
#pragma unroll
            for (int k = 0; k < kM; ++k) {
                float fr = __shfl_down_sync(0xffffffffu, acc[0][k + 1], 1);  // from column x + 1
                float fl = __shfl_up_sync(0xffffffffu, acc[2][k + 1], 1);    // from column x - 1
                if (lane == 31) fr = (x == 31) ? sm.er2l[ex][strip][k] : 0.0f;
                if (lane == 0) fl = (x == 32) ? sm.el2r[ex][strip][k] : 0.0f;
                float v = fmaf(pc, lb[k], acc[1][k + 1] + fr + fl);
                if (k == 0 && strip > 0) {
                    v += sm.vbot[ex][strip - 1][1][x];
                    if (x + 1 < kCT) v += sm.vbot[ex][strip - 1][0][x + 1];
                    if (x >= 1) v += sm.vbot[ex][strip - 1][2][x - 1];
                }
                if (k == kM - 1 && strip < kStrips - 1) {
                    v += sm.vtop[ex][strip + 1][1][x];
                    if (x + 1 < kCT) v += sm.vtop[ex][strip + 1][0][x + 1];
                    if (x >= 1) v += sm.vtop[ex][strip + 1][2][x - 1];
                }
                lb[k] = v;
            }
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
#pragma unroll
                for (int d = 0; d < 8; ++d) Gq[d * gplane + j] += gv[d];
            }
        }
    }
    if (failed && tid == 0) {
        atomicExch(err, kErrTmaTimeout);
        // give the copies in flight one more bounded wait before the CTA exits
        mbar_wait_bounded(&qbar, 0);
        mbar_wait_bounded(&sbar[0], 0);
        mbar_wait_bounded(&sbar[1], 0);
    }
    tmem_sync_threads();
    if (warp == 0) tmem_dealloc(tslot, kTmemCols);
}

}  // namespace

int adjoint_blocked_max_steps() { return kMaxSteps; }

static size_t adjoint_blocked_smem() { return sizeof(Smem) + 128; }

int adjoint_blocked_configure() {
    static int done = 0;
    if (!done) {
        if (cudaFuncSetAttribute(k_adjoint_blocked, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)adjoint_blocked_smem()) != cudaSuccess)
            return -1;
        done = 1;
    }
    return 0;
}

void launch_adjoint_blocked(const CUtensorMap* tst, const CUtensorMap* tq, int H, int pitch, float pc, int zlast,
                            int n, const float* lam_in, float* lam_out, float* Gq, int nsm, int* err, cudaStream_t s) {
    const int tiles_x = (pitch + kIC - 1) / kIC;
    const int tiles_y = (H + kIR - 1) / kIR;
    const int ntiles = tiles_x * tiles_y;
    const int grid = ntiles < nsm ? ntiles : nsm;
    k_adjoint_blocked<<<grid, kThreads, adjoint_blocked_smem(), s>>>(*tst, *tq, H, pitch, pc, zlast, n, tiles_x,
                                                                     ntiles, lam_in, lam_out, Gq, err);
}

}  // namespace pf
