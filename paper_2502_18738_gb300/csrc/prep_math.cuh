// The per-cell fold of Eq. 1-5 (the prep's arithmetic), shared by the prep kernel and
// the step kernels that recompute q instead of reading it, so that both give the same
// bits. Internal to libpfire.
#pragma once
#include "common.cuh"

namespace pf {

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

// q[d] of cell (r, c) for the 8 directions (0 for a non-burnable cell and for
// neighbours outside the grid): the values k_prep stores.
__device__ __forceinline__ void q_cell(const PrepArgs& g, int r, int c, float (&q)[8]) {
    if (g.burnable && g.burnable[(size_t)r * g.W + c] == 0) {
#pragma unroll
        for (int d = 0; d < 8; ++d) q[d] = 0.0f;
        return;
    }
    const CellFactors f = load_cell(g, r, c);
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        float expo, ts, cm1;
        q[d] = dir_exponent(g, f, r, c, d, expo, ts, cm1) ? q_of(f, expf(expo), nullptr) : 0.0f;  // Eq. 2, 5
    }
}

}  // namespace pf
