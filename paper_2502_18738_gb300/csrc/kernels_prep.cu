// Prep (Eq. 1-5): fold the static landscape, the wind epoch and the parameters into
// eight per-cell directional ignition factors q[d][r][c] = f_p(p_propagate), and the
// chain rule of that fold for the adjoint.
#include <cmath>

#include "common.cuh"
#include "prep_math.cuh"

namespace pf {

namespace {

__global__ void __launch_bounds__(256) k_prep(PrepArgs g, float* __restrict__ q) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= g.H || c >= g.pitch) return;
    // outside the reach mask (and in the padding columns, which hold zeros) q is not read
    // where it matters: keep what the buffer holds
    if (g.reach && (c >= g.W || !g.reach[(r >> 5) * g.reach_bw + (c >> 5)])) return;
    const size_t plane = (size_t)g.H * g.pitch;
    float* qo = q + (size_t)r * g.pitch + c;
    float qv[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    if (c < g.W) q_cell(g, r, c, qv);
#pragma unroll
    for (int d = 0; d < 8; ++d) qo[d * plane] = qv[d];
}

// One warp per 32 x 32 block, a lane per column: whether any a or b bit is set (b's sign
// bit ignored, as -0 is no fire).
__global__ void __launch_bounds__(256) k_reach_any(const float* __restrict__ ab, int H, int W, int pitch, int bw,
                                                   int nblk, uint8_t* __restrict__ any) {
    const int b = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (b >= nblk) return;
    const int r0 = (b / bw) * 32, c = (b % bw) * 32 + lane;
    const int r1 = min(r0 + 32, H);
    const size_t plane = (size_t)H * pitch;
    uint32_t v = 0u;
    if (c < W)
        for (int r = r0; r < r1; ++r) {
            v |= __float_as_uint(__ldg(ab + (size_t)r * pitch + c));
            v |= __float_as_uint(__ldg(ab + plane + (size_t)r * pitch + c)) & 0x7fffffffu;
        }
    const bool hit = __any_sync(0xffffffffu, v != 0u);
    if (lane == 0) any[b] = hit ? 1 : 0;
}

// One pass of a separable block dilation: out[B] = OR of in over the blocks within
// `radius` of B along rows (horizontal) or columns.
__global__ void __launch_bounds__(256) k_reach_dilate(const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                                                      int bh, int bw, int radius, int horizontal) {
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= bh * bw) return;
    const int by = i / bw, bx = i % bw;
    uint8_t v = 0;
    for (int k = -radius; k <= radius && !v; ++k) {
        const int y = horizontal ? by : by + k, x = horizontal ? bx + k : bx;
        if (y >= 0 && y < bh && x >= 0 && x < bw) v = in[y * bw + x];
    }
    out[i] = v;
}

// acc[B] |= in[B] over nb bytes
__global__ void __launch_bounds__(256) k_reach_or(uint8_t* __restrict__ acc, const uint8_t* __restrict__ in, int nb) {
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i < nb) acc[i] |= in[i];
}

constexpr int kAdjThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// One thread per cell (grid-stride, fixed assignment): the parameter partials are
// accumulated per thread in FP32 over the 8 directions of a cell and in FP64 across
// cells, reduced by warp shuffles and then across the block, and written as one FP64
// row per block. Per-cell gradients are accumulated into gpveg / gpden.
__global__ void __launch_bounds__(kAdjThreads) k_prep_adjoint(PrepArgs g, float* __restrict__ Gq,
                                                              double* __restrict__ partials,
                                                              float* __restrict__ gpveg,
                                                              float* __restrict__ gpden) {
    const size_t plane = (size_t)g.H * g.pitch;
    const size_t HW = (size_t)g.H * g.W;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (size_t j = (size_t)blockIdx.x * kAdjThreads + threadIdx.x; j < HW; j += (size_t)gridDim.x * kAdjThreads) {
        const int r = (int)(j / g.W), c = (int)(j % g.W);
        if (g.gq_dirty && !g.gq_dirty[(r / 48) * g.gq_tiles_x + c / 48]) continue;  // dL/dq = 0 here
        float* gq = Gq + (size_t)r * g.pitch + c;
        // cells no fire reached during the epoch have dL/dq = 0 in every direction and
        // contribute nothing: skip their (transcendental-heavy) derivative evaluation.
        // The others are cleared for the next epoch here, so that Gq is all zeros again
        // after the pass without a separate sweep over it.
        float gqv[8];
        bool any = false;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            gqv[d] = gq[d * plane];
            any |= gqv[d] != 0.0f;
        }
        if (!any) continue;
#pragma unroll
        for (int d = 0; d < 8; ++d) gq[d * plane] = 0.0f;
        if (g.burnable && g.burnable[j] == 0) continue;
        const CellFactors f = load_cell(g, r, c);
        float sh = 0.f, s1 = 0.f, s2 = 0.f, sa = 0.f, se = 0.f;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            float expo, ts, cm1;
            if (!dir_exponent(g, f, r, c, d, expo, ts, cm1)) continue;
            const float e = expf(expo);
            float pp;
            const float qq = q_of(f, e, &pp);
            const float gpp = gqv[d] * kC * ((1.0f - qq) * (1.0f + qq));  // tanh'
            se += gpp * e;              // d pp / d(p_h (1+pv)(1+pd)) summed over d
            sh += gpp * f.G * e;        // d pp / d p_h
            s1 += gpp * pp * f.V;       // d pp / d c1
            s2 += gpp * pp * f.V * cm1; // d pp / d c2
            sa += gpp * pp * ts;        // d pp / d a
        }
        acc[0] += sh; acc[1] += s1; acc[2] += s2; acc[3] += sa;
        if (gpveg) gpveg[j] += se * g.p_h * (1.0f + f.pd);
        if (gpden) gpden[j] += se * g.p_h * (1.0f + f.pv);
    }
    __shared__ double red[kAdjThreads / 32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double v = warp_sum(acc[k]);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int w = 0; w < kAdjThreads / 32; ++w) s += red[w][threadIdx.x];
        partials[(size_t)blockIdx.x * 4 + threadIdx.x] = s;
    }
}

constexpr int kRedThreads = 512;

// Fixed-order FP64 sum of the block partials: thread t sums rows t, t+512, ... in order,
// then a fixed shuffle/shared-memory tree; bit-reproducible for a given nblk.
__global__ void __launch_bounds__(kRedThreads) k_reduce_partials(const double* __restrict__ partials, int nblk,
                                                                 double* __restrict__ acc) {
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblk; b += kRedThreads)
#pragma unroll
        for (int k = 0; k < 4; ++k) s[k] += partials[(size_t)b * 4 + k];
    __shared__ double red[kRedThreads / 32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double v = warp_sum(s[k]);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) t += red[w][threadIdx.x];
        acc[threadIdx.x] += t;
    }
}

}  // namespace

static void split(double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

void prep_derive(PrepArgs& g) {
    const double pi = 3.14159265358979323846;
    split((double)g.a * (180.0 / pi), g.adeg_hi, g.adeg_lo);
    split(1.0 / (double)g.l, g.ikl_e_hi, g.ikl_e_lo);
    split(1.0 / (std::sqrt(2.0) * (double)g.l), g.ikl_d_hi, g.ikl_d_lo);
}

int prep_reach_bytes(int H, int W) { return ((H + 31) / 32) * ((W + 31) / 32); }

void launch_prep_reach(const float* ab, int H, int W, int pitch, int radius, uint8_t* tmp, uint8_t* reach,
                       cudaStream_t s) {
    const int bh = (H + 31) / 32, bw = (W + 31) / 32, nb = bh * bw;
    k_reach_any<<<(nb + 7) / 8, 256, 0, s>>>(ab, H, W, pitch, bw, nb, reach);
    k_reach_dilate<<<(nb + 255) / 256, 256, 0, s>>>(reach, tmp, bh, bw, radius, 1);
    k_reach_dilate<<<(nb + 255) / 256, 256, 0, s>>>(tmp, reach, bh, bw, radius, 0);
}

void launch_reach_or(uint8_t* acc, const uint8_t* in, int nb, cudaStream_t s) {
    if (nb > 0) k_reach_or<<<(nb + 255) / 256, 256, 0, s>>>(acc, in, nb);
}

void launch_prep(const PrepArgs& g, float* q, cudaStream_t s) {
    dim3 blk(64, 4);
    dim3 grd((g.pitch + blk.x - 1) / blk.x, (g.H + blk.y - 1) / blk.y);
    k_prep<<<grd, blk, 0, s>>>(g, q);
}

int prep_adjoint_blocks(int H, int W) {
    const size_t HW = (size_t)H * W;
    size_t want = (HW + kAdjThreads - 1) / kAdjThreads;
    const size_t cap = 152 * 8;  // 8 resident blocks per SM on 152 SMs
    return (int)(want < cap ? (want ? want : 1) : cap);
}

void launch_prep_adjoint(const PrepArgs& g, float* Gq, double* partials, float* gpveg, float* gpden,
                         cudaStream_t s) {
    const int nblk = prep_adjoint_blocks(g.H, g.W);
    k_prep_adjoint<<<nblk, kAdjThreads, 0, s>>>(g, Gq, partials, gpveg, gpden);
}

void launch_reduce_partials(const double* partials, int nblk, double* acc, cudaStream_t s) {
    k_reduce_partials<<<1, kRedThreads, 0, s>>>(partials, nblk, acc);
}

}  // namespace pf
