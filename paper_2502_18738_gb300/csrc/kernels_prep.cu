// Prep (Eq. 1-5): fold the static landscape, the wind epoch and the parameters into
// eight per-cell directional ignition factors q[d][r][c] = f_p(p_propagate), and the
// chain rule of that fold for the adjoint.
#include <cmath>

#include "common.cuh"

namespace pf {

namespace {

// Systematic rounding of a constant shared by every cell (c, 180/pi, sqrt 2, 1 + p_veg
// of one vegetation class) biases q the same way in every cell, and such a bias
// compounds along a fire path of D cells into a relative error ~D times larger in the
// state. So the constants and the products of the fold are carried as unevaluated
// float pairs (hi + lo, Dekker/Knuth error-free transformations with FMA); only the
// transcendental calls (atan, exp, tanh, sincospi) run in plain FP32, whose errors
// vary from cell to cell and average out along a path.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ DF df_mul_f(DF x, float y) {
    const float p = x.hi * y;
    return {p, fmaf(x.lo, y, fmaf(x.hi, y, -p))};
}
__device__ __forceinline__ DF df_mul(DF x, DF y) {
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return {p, e};
}
__device__ __forceinline__ float df_times(float x, float hi, float lo) { return fmaf(x, hi, x * lo); }

// c of Eq. 8 as hi + lo
constexpr float kChi = 1.1486328125f;
constexpr float kClo = (float)(1.1486328125 - (double)kChi);
// sqrt(2)/2 as hi + lo
constexpr float kRhi = 0.70710678118654752f;
constexpr float kRlo = (float)(0.70710678118654752440 - (double)kRhi);
constexpr float kRadToDeg = 57.295779513082320876f;

// Direction of travel from the burning neighbour to the receiving cell, counter-
// clockwise from East (north = decreasing row): phi_d = atan2(dr, -dc). cos(theta_w -
// phi_d) = cos(theta_w) cos(phi_d) + sin(theta_w) sin(phi_d) with (cos, sin) of phi_d
// in {0, +-1, +-sqrt(2)/2}: stored as signs, the diagonal factor applied in hi + lo.
__device__ __forceinline__ float cos_rel(int d, float cw, float sw) {
    switch (d) {
        case 0: { const float u = cw - sw; return df_times(u, kRhi, kRlo); }   // phi = -45
        case 1: return -sw;                                                     // phi = -90
        case 2: { const float u = -cw - sw; return df_times(u, kRhi, kRlo); }  // phi = -135
        case 3: return cw;                                                      // phi = 0
        case 4: return -cw;                                                     // phi = 180
        case 5: { const float u = cw + sw; return df_times(u, kRhi, kRlo); }   // phi = 45
        case 6: return sw;                                                      // phi = 90
        default: { const float u = sw - cw; return df_times(u, kRhi, kRlo); }  // phi = 135
    }
}

struct CellFactors {
    DF Gp;        // p_h (1 + p_veg)(1 + p_den)
    float G;      // (1 + p_veg)(1 + p_den), FP32
    float V;      // wind speed
    float cw, sw; // cos / sin of the wind direction
    float pv, pd;
    float Ej;
};

__device__ __forceinline__ CellFactors load_cell(const PrepArgs& g, int r, int c) {
    const size_t j = (size_t)r * g.W + c;
    CellFactors f;
    f.pv = g.pveg ? g.pveg[j] : 0.0f;
    f.pd = g.pden ? g.pden[j] : 0.0f;
    const DF g1 = two_sum(1.0f, f.pv), g2 = two_sum(1.0f, f.pd);
    const DF G = df_mul(g1, g2);
    f.Gp = df_mul_f(G, g.p_h);
    f.G = G.hi + G.lo;
    f.V = g.V ? g.V[j] : 0.0f;
    const float th = g.th ? g.th[j] : 0.0f;
    sincospif(th * (1.0f / 180.0f), &f.sw, &f.cw);
    f.Ej = g.E ? g.E[j] : 0.0f;
    return f;
}

// Exponent of p_w * p_s (Eq. 3 and 4 combined) for direction d; false when the
// neighbour lies outside the grid. Also returns theta_s (deg) and cos(theta) - 1.
__device__ __forceinline__ bool dir_exponent(const PrepArgs& g, const CellFactors& f, int r, int c, int d,
                                             float& expo, float& theta_s, float& cosm1) {
    const int ri = r + dir_dr(d), ci = c + dir_dc(d);
    if (ri < 0 || ri >= g.H || ci < 0 || ci >= g.W) return false;
    cosm1 = cos_rel(d, f.cw, f.sw) - 1.0f;
    float slope_term;
    if (g.slope) {
        // the H x W x 3 x 3 slope input (Sec. 2.1), degrees, [r][c][dr+1][dc+1]
        theta_s = g.slope[((size_t)r * g.W + c) * 9 + (dir_dr(d) + 1) * 3 + (dir_dc(d) + 1)];
        slope_term = g.a * theta_s;
    } else {
        float dE = 0.0f;
        if (g.E) dE = f.Ej - g.E[(size_t)ri * g.W + ci];
        const bool diag = (dir_dr(d) != 0) && (dir_dc(d) != 0);
        const float x = diag ? df_times(dE, g.ikl_d_hi, g.ikl_d_lo) : df_times(dE, g.ikl_e_hi, g.ikl_e_lo);
        const float t = atanf(x);                                       // Eq. 1, radians
        theta_s = t * kRadToDeg;
        slope_term = df_times(t, g.adeg_hi, g.adeg_lo);                 // a theta_s(deg), a*180/pi as hi + lo
    }
    // Eq. 3 x Eq. 4 exponent: c1 V + c2 V (cos - 1) + a theta_s
    expo = fmaf(g.c2 * f.V, cosm1, fmaf(g.c1, f.V, slope_term));
    return true;
}

// q = tanh(c pp), pp = p_h (1+pv)(1+pd) e, with the products in hi + lo.
__device__ __forceinline__ float q_of(const CellFactors& f, float e, float* pp_out) {
    const DF pp = df_mul_f(f.Gp, e);
    const DF y = df_mul(pp, DF{kChi, kClo});
    const float th = tanhf(y.hi);
    if (pp_out) *pp_out = pp.hi + pp.lo;
    return fmaf((1.0f - th) * (1.0f + th), y.lo, th);
}

__global__ void __launch_bounds__(256) k_prep(PrepArgs g, float* __restrict__ q) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= g.H || c >= g.pitch) return;
    // outside the reach mask (and in the padding columns, which hold zeros) q is not read
    // where it matters: keep what the buffer holds
    if (g.reach && (c >= g.W || !g.reach[(r >> 5) * g.reach_bw + (c >> 5)])) return;
    const size_t plane = (size_t)g.H * g.pitch;
    float* qo = q + (size_t)r * g.pitch + c;
    if (c >= g.W || (g.burnable && g.burnable[(size_t)r * g.W + c] == 0)) {
#pragma unroll
        for (int d = 0; d < 8; ++d) qo[d * plane] = 0.0f;
        return;
    }
    const CellFactors f = load_cell(g, r, c);
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        float expo, ts, cm1, v = 0.0f;
        if (dir_exponent(g, f, r, c, d, expo, ts, cm1)) v = q_of(f, expf(expo), nullptr);  // Eq. 2, 5
        qo[d * plane] = v;
    }
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
