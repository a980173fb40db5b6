// Differentiable (mean-field) step and its reverse-time adjoint.
// State (a, b) = (P[ever ignited], P[burning]) as two FP32 planes [2][H][pitch], a held
// in the complement-aware encoding A (common.cuh):
//   P_j  = 1 - prod_d (1 - b_{j+d} q_dj)     (Eq. 9 with burning probabilities)
//   n_j  = (1 - a_j) P_j,  a'_j = a_j + n_j,  b'_j = n_j + p_continue b_j
// P is accumulated as P <- P + x (1 - P), which keeps small probabilities accurate in
// FP32, and the survival product S = prod_d (1 - x_d) alongside it, so that
// 1 - a' = (1 - a) S is formed without cancellation.
#include "common.cuh"
#include "prep_math.cuh"

namespace pf {

namespace {

__global__ void __launch_bounds__(256) k_diff_step(int H, int W, int pitch, float pc, const float* __restrict__ ab,
                                                   float* __restrict__ abn, const float* __restrict__ q) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= H || c >= pitch) return;
    const size_t plane = (size_t)H * pitch;
    const size_t j = (size_t)r * pitch + c;
    if (c >= W) {
        abn[j] = 0.0f;
        abn[plane + j] = 0.0f;
        return;
    }
    float nb[8], qv[8];
    int nk[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const int ri = r + dir_dr(d), ci = c + dir_dc(d);
        const bool in = ri >= 0 && ri < H && ci >= 0 && ci < W;
        const size_t i = in ? (size_t)ri * pitch + ci : j;
        float Ai, Bi;
        x_decode(__ldg(ab + i), __ldg(ab + plane + i), Ai, Bi, nk[d]);
        nb[d] = in ? Bi : 0.0f;
        qv[d] = __ldg(q + d * plane + j);
    }
    float A, B, An, Bn;
    int k, kn;
    x_decode(ab[j], ab[plane + j], A, B, k);
    x_update(nb, nk, qv, A, B, k, pc, An, Bn, kn);
    x_encode(An, Bn, kn, abn[j], abn[plane + j]);
}

// The same step with q recomputed from the fields in every cell and step (prep's
// arithmetic, q_cell) instead of read from the materialised planes: the same bits.
__global__ void __launch_bounds__(256) k_diff_step_rc(PrepArgs g, float pc, const float* __restrict__ ab,
                                                      float* __restrict__ abn) {
    const int H = g.H, W = g.W, pitch = g.pitch;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= H || c >= pitch) return;
    const size_t plane = (size_t)H * pitch;
    const size_t j = (size_t)r * pitch + c;
    if (c >= W) {
        abn[j] = 0.0f;
        abn[plane + j] = 0.0f;
        return;
    }
    float nb[8], qv[8];
    int nk[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const int ri = r + dir_dr(d), ci = c + dir_dc(d);
        const bool in = ri >= 0 && ri < H && ci >= 0 && ci < W;
        const size_t i = in ? (size_t)ri * pitch + ci : j;
        float Ai, Bi;
        x_decode(__ldg(ab + i), __ldg(ab + plane + i), Ai, Bi, nk[d]);
        nb[d] = in ? Bi : 0.0f;
    }
    q_cell(g, r, c, qv);
    float A, B, An, Bn;
    int k, kn;
    x_decode(ab[j], ab[plane + j], A, B, k);
    x_update(nb, nk, qv, A, B, k, pc, An, Bn, kn);
    x_encode(An, Bn, kn, abn[j], abn[plane + j]);
}

// p_ignite of every cell (FP32; values below FP32's range read as 0)
__global__ void k_ignition_map_diff(int H, int W, int pitch, const float* __restrict__ ab,
                                    const float* __restrict__ q, float* __restrict__ Pout) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)H * W) return;
    const int r = (int)(idx / W), c = (int)(idx % W);
    const size_t plane = (size_t)H * pitch;
    const size_t j = (size_t)r * pitch + c;
    float nb[8];
    int nk[8];
    int kP = kKNone;
    for (int d = 0; d < 8; ++d) {
        const int ri = r + dir_dr(d), ci = c + dir_dc(d);
        const bool in = ri >= 0 && ri < H && ci >= 0 && ci < W;
        const size_t i = in ? (size_t)ri * pitch + ci : j;
        float Ai;
        x_decode(ab[i], ab[plane + i], Ai, nb[d], nk[d]);
        nb[d] = in ? nb[d] : 0.0f;
        nk[d] = nb[d] != 0.0f ? nk[d] : kKNone;  // the b-tier
        kP = min(kP, nk[d]);
    }
    float P = 0.0f, S = 1.0f;
    for (int d = 0; d < 8; ++d) {
        const float x = __fmul_rn(__fmul_rn(nb[d], q[d * plane + j]), tier_scale(nk[d] - kP));
        P = fmaf(x, S, P);
        S = kP == 0 ? fmaf(-x, S, S) : S;
    }
    Pout[idx] = P * tier_scale(kP);
}

// ---------------------------------------------------------------- adjoint
// Reverse-mode transpose of k_diff_step for one step. With lambda' = dL/d(a', b'):
//   l_n = l_a'_j + l_b'_j,  l_a_j = l_a'_j - l_n P_j,  l_P_j = l_n (1 - a_j)
//   l_b_i = p_c l_b'_i + sum_{targets j of i} l_P_j q_dj prod_{e != d} (1 - b_e q_ej)
//   Gq_dj += l_P_j b_{j+d} prod_{e != d} (1 - b_e q_ej)
// in the scaled form of common.cuh (lambda = mu 2^sigma). The leave-one-out products
// come from prefix / suffix products (no division, since a factor 1 - b q can be exactly
// 0). Each block computes the per-target contributions of its tile plus a one-cell ring
// into shared memory, then gathers them per source cell.
constexpr int kAX = 32, kAY = 8;

__global__ void __launch_bounds__(kAX * kAY) k_adjoint_step(int H, int W, int pitch, float pc,
                                                            const float* __restrict__ ab,
                                                            const float* __restrict__ q,
                                                            const float* __restrict__ lam1,
                                                            const uint8_t* __restrict__ sig1,
                                                            float* __restrict__ lam0, uint8_t* __restrict__ sig0,
                                                            float* __restrict__ Gq) {
    __shared__ float sbt[kAY + 4][kAX + 4];         // true b at t (FP32, tiers flushed), rows r0-2 .. r0+kAY+1
    __shared__ float sbs[kAY + 4][kAX + 4];         // b at t in its tier's units, b 2^(64 sigma)
    __shared__ int ssg[kAY + 4][kAX + 4];           // sigma(t) of the same cells (the tier)
    __shared__ float sc[8][kAY + 2][kAX + 2];       // contributions of targets j, in source units
    const int c0 = blockIdx.x * kAX, r0 = blockIdx.y * kAY;
    const int tid = threadIdx.y * kAX + threadIdx.x;
    const size_t plane = (size_t)H * pitch;
    const float* a = ab;
    const float* b = ab + plane;
    const float* la1 = lam1;
    const float* lb1 = lam1 + plane;
    for (int i = tid; i < (kAY + 4) * (kAX + 4); i += kAX * kAY) {
        const int y = i / (kAX + 4), x = i % (kAX + 4);
        const int r = r0 - 2 + y, c = c0 - 2 + x;
        const bool in = r >= 0 && r < H && c >= 0 && c < W;
        float bt = 0.0f, bs = 0.0f;
        int sg = kSigmaZero;
        if (in) {
            const float As = a[(size_t)r * pitch + c], Bs = b[(size_t)r * pitch + c];
            float A, B;
            int k;
            x_decode(As, Bs, A, B, k);
            sg = x_sigma(As, Bs);
            bt = B * tier_scale(k);
            bs = B;
        }
        sbt[y][x] = bt;
        sbs[y][x] = bs;
        ssg[y][x] = sg;
    }
    __syncthreads();
    for (int i = tid; i < (kAY + 2) * (kAX + 2); i += kAX * kAY) {
        const int y = i / (kAX + 2), x = i % (kAX + 2);
        const int r = r0 - 1 + y, c = c0 - 1 + x;
        const size_t j = (size_t)r * pitch + c;
        const int sgp = (r >= 0 && r < H && c >= 0 && c < W) ? __ldg(sig1 + j) : kSigmaZero;
        if (sgp == kSigmaZero) {  // outside the grid, or a = 0 at t + 1 (so also at t)
#pragma unroll
            for (int d = 0; d < 8; ++d) sc[d][y][x] = 0.0f;
            continue;
        }
        float qd[8], f[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            qd[d] = __ldg(q + d * plane + j);
            f[d] = fmaf(-sbt[y + 1 + dir_dr(d)][x + 1 + dir_dc(d)], qd[d], 1.0f);
        }
        float pre[8], suf[8];
        pre[0] = 1.0f;
#pragma unroll
        for (int d = 1; d < 8; ++d) pre[d] = pre[d - 1] * f[d - 1];
        suf[7] = 1.0f;
#pragma unroll
        for (int d = 6; d >= 0; --d) suf[d] = suf[d + 1] * f[d + 1];
        const float P = 1.0f - pre[7] * f[7];
        const float la = __ldg(la1 + j), lb = __ldg(lb1 + j);
        const float ln = la + lb;
        const float As = __ldg(a + j);
        // 1 - a: 1 for a tiered cell (a < 2^-64)
        const float ua = signbit(As) ? -As : (x_tier(As, __ldg(b + j)) == 0 ? 1.0f - As : 1.0f);
        const float tg = ln * ua;  // l_P_j in units 2^(64 sigma'(j))
        const bool interior = (y >= 1 && y <= kAY && x >= 1 && x <= kAX);
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const int yy = y + 1 + dir_dr(d), xx = x + 1 + dir_dc(d);
            const float t = tg * (pre[d] * suf[d]);
            const float r_d = exp2i(64 * (sgp - ssg[yy][xx]));  // 2^(64 (sigma'(j) - sigma(i)))
            sc[d][y][x] = t * qd[d] * r_d;
            if (interior) Gq[d * plane + j] = fmaf(t, sbs[yy][xx] * r_d, Gq[d * plane + j]);
        }
        if (interior) lam0[j] = fmaf(-ln, P, la) * exp2i(64 * (sgp - ssg[y + 1][x + 1]));
    }
    __syncthreads();
    const int x = threadIdx.x, y = threadIdx.y;
    const int r = r0 + y, c = c0 + x;
    if (r >= H || c >= W) return;
    const size_t j = (size_t)r * pitch + c;
    const int sgp = __ldg(sig1 + j);
    const int sg = ssg[y + 2][x + 2];
    float acc = 0.0f;
    if (sgp != kSigmaZero) acc = pc * __ldg(lb1 + j) * exp2i(64 * (sgp - sg));
#pragma unroll
    for (int d = 0; d < 8; ++d) acc += sc[d][y + 1 - dir_dr(d)][x + 1 - dir_dc(d)];  // target j = i - offset
    if (sg == kSigmaZero || sgp == kSigmaZero) {  // a == 0 at t: lambda multiplies only zeros
        acc = 0.0f;
        lam0[j] = 0.0f;
    }
    lam0[plane + j] = acc;
    sig0[j] = (uint8_t)sg;
}

__global__ void k_adjoint_init(const float* __restrict__ dLda, const float* __restrict__ dLdb,
                               const float* __restrict__ ab, int H, int W, int pitch, float* __restrict__ lam,
                               uint8_t* __restrict__ sig) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= H || c >= pitch) return;
    const size_t plane = (size_t)H * pitch;
    const size_t j = (size_t)r * pitch + c;
    float la = 0.0f, lb = 0.0f;
    int sg = kSigmaZero;
    if (c < W) {
        sg = x_sigma(ab[j], ab[plane + j]);
        if (sg != kSigmaZero) {
            const float ui = exp2i(-64 * sg);
            if (dLda) la = dLda[(size_t)r * W + c] * ui;
            if (dLdb) lb = dLdb[(size_t)r * W + c] * ui;
        }
    }
    lam[j] = la;
    lam[plane + j] = lb;
    sig[j] = (uint8_t)sg;
}

}  // namespace

void launch_diff_step(int H, int W, int pitch, float pc, const float* ab, float* abn, const float* q,
                      cudaStream_t s) {
    dim3 blk(64, 4);
    dim3 grd((pitch + 63) / 64, (H + 3) / 4);
    k_diff_step<<<grd, blk, 0, s>>>(H, W, pitch, pc, ab, abn, q);
}

void launch_diff_step_rc(const PrepArgs& g, float pc, const float* ab, float* abn, cudaStream_t s) {
    dim3 blk(64, 4);
    dim3 grd((g.pitch + 63) / 64, (g.H + 3) / 4);
    k_diff_step_rc<<<grd, blk, 0, s>>>(g, pc, ab, abn);
}

void launch_ignition_map_diff(int H, int W, int pitch, const float* ab, const float* q, float* P, cudaStream_t s) {
    const size_t n = (size_t)H * W;
    k_ignition_map_diff<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(H, W, pitch, ab, q, P);
}

void launch_adjoint_step(int H, int W, int pitch, float pc, const float* ab, const float* q, const float* lam1,
                         const uint8_t* sig1, float* lam0, uint8_t* sig0, float* Gq, cudaStream_t s) {
    dim3 blk(kAX, kAY);
    dim3 grd((W + kAX - 1) / kAX, (H + kAY - 1) / kAY);
    k_adjoint_step<<<grd, blk, 0, s>>>(H, W, pitch, pc, ab, q, lam1, sig1, lam0, sig0, Gq);
}

void launch_adjoint_init(const float* dLda, const float* dLdb, const float* ab, int H, int W, int pitch, float* lam,
                         uint8_t* sig, cudaStream_t s) {
    dim3 blk(64, 4);
    dim3 grd((pitch + 63) / 64, (H + 3) / 4);
    k_adjoint_init<<<grd, blk, 0, s>>>(dLda, dLdb, ab, H, W, pitch, lam, sig);
}

}  // namespace pf
