// Small helper kernels: input validation, continuous-state initialisation, and the
// binary cross-entropy loss of a burn-probability map.
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace pf {

namespace {

__global__ void k_validate_fields(const float* __restrict__ x, size_t n, float lo, int bit, int* flags) {
    bool bad = false;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float v = x[i];
        bad |= !isfinite(v) || v < lo;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, 1 << bit);
}

__global__ void k_validate_states(const uint8_t* __restrict__ S, size_t n, int* flags) {
    bool bad = false;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        bad |= S[i] > 3;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, 1);
}

// a = [S in {2,3}], b = [S == 2]; burnable = [S != 0]
__global__ void k_diff_init(const uint8_t* __restrict__ S, int H, int W, int pitch, float* __restrict__ ab,
                            uint8_t* __restrict__ burn) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)H * W) return;
    const int r = (int)(idx / W), c = (int)(idx % W);
    const uint8_t s = S[idx];
    const size_t j = (size_t)r * pitch + c;
    ab[j] = (s == 2 || s == 3) ? -0.0f : 0.0f;  // encoded a: -0.0 is a = 1
    ab[(size_t)H * pitch + j] = (s == 2) ? 1.0f : 0.0f;
    burn[idx] = s != 0;
}

__global__ void k_diff_pack(const float* __restrict__ dense, int H, int W, int pitch, float* __restrict__ ab) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t HW = (size_t)H * W;
    if (idx >= HW) return;
    const int r = (int)(idx / W), c = (int)(idx % W);
    const size_t j = (size_t)r * pitch + c;
    const float a = dense[idx], b = dense[HW + idx];
    // values below 2^-64 go to their tier; b = -0 is stored as +0 (the sign marks a tier)
    float A = a_encode(a, 1.0f - a), B = b <= 0.0f ? 0.0f : b;
    int k = 0;
    x_renorm(A, B, k);
    x_encode(A, B, k, ab[j], ab[(size_t)H * pitch + j]);
}

// Cells in each state 0..3 over all realisations (grid-stride; one atomic per block and state).
__global__ void __launch_bounds__(256) k_state_counts(const uint8_t* __restrict__ S, int R, int H, int W, int pitch,
                                                      unsigned long long* __restrict__ counts) {
    __shared__ unsigned long long sc[4];
    if (threadIdx.x < 4) sc[threadIdx.x] = 0ull;
    __syncthreads();
    unsigned long long c[4] = {0ull, 0ull, 0ull, 0ull};
    const size_t n = (size_t)R * H * W;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t rr = i / ((size_t)H * W), j = i % ((size_t)H * W);
        const uint8_t v = S[(rr * H + j / W) * pitch + j % W];
        c[v & 3u] += 1ull;
    }
    for (int k = 0; k < 4; ++k)
        if (c[k]) atomicAdd(&sc[k], c[k]);
    __syncthreads();
    if (threadIdx.x < 4 && sc[threadIdx.x]) atomicAdd(counts + threadIdx.x, sc[threadIdx.x]);
}

// Burnable cells, and FP64 sums of a and b over the grid (tiers below FP32's range add 0).
__global__ void __launch_bounds__(256) k_diff_sums(const float* __restrict__ ab, const uint8_t* __restrict__ burn,
                                                   int H, int W, int pitch, unsigned long long* __restrict__ nburn,
                                                   double* __restrict__ sums) {
    __shared__ double s2[2][8];
    __shared__ unsigned long long sn[8];
    double sa = 0.0, sb = 0.0;
    unsigned long long nb = 0ull;
    const size_t n = (size_t)H * W, plane = (size_t)H * pitch;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t j = (i / W) * pitch + i % W;
        float A, B;
        int k;
        x_decode(ab[j], ab[plane + j], A, B, k);
        sa += signbit(A) ? 1.0 + (double)A : (double)(A * tier_scale(k));
        sb += (double)(B * tier_scale(k));
        nb += burn && burn[i] ? 1ull : 0ull;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_down_sync(0xffffffffu, sa, o);
        sb += __shfl_down_sync(0xffffffffu, sb, o);
        nb += __shfl_down_sync(0xffffffffu, nb, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s2[0][w] = sa;
        s2[1][w] = sb;
        sn[w] = nb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        unsigned long long tn = 0ull;
        for (int k = 0; k < 8; ++k) {
            ta += s2[0][k];
            tb += s2[1][k];
            tn += sn[k];
        }
        atomicAdd(sums, ta);
        atomicAdd(sums + 1, tb);
        atomicAdd(nburn, tn);
    }
}

__global__ void k_diff_unpack(const float* __restrict__ ab, int H, int W, int pitch, float* __restrict__ dense) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t HW = (size_t)H * W;
    if (idx >= HW) return;
    const int r = (int)(idx / W), c = (int)(idx % W);
    const size_t j = (size_t)r * pitch + c;
    float A, B;
    int k;
    x_decode(ab[j], ab[(size_t)H * pitch + j], A, B, k);
    // plain FP32: values of the tiers below FP32's range read as 0
    dense[idx] = signbit(A) ? 1.0f + A : A * tier_scale(k);
    dense[HW + idx] = B * tier_scale(k);
}

constexpr int kBceThreads = 256;
constexpr float kBceEps = 1e-7f;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kBceThreads) k_bce(const float* __restrict__ a, const float* __restrict__ y,
                                                     int64_t n, float* __restrict__ g, double* __restrict__ partials) {
    double acc = 0.0;
    const float inv_n = (float)(1.0 / (double)n);
    for (int64_t i = (int64_t)blockIdx.x * kBceThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBceThreads) {
        const float av = a[i], yv = y[i];
        const float yh = fminf(fmaxf(av, kBceEps), 1.0f - kBceEps);
        acc -= (double)(yv * logf(yh) + (1.0f - yv) * logf(1.0f - yh));
        if (g) g[i] = (av >= kBceEps && av <= 1.0f - kBceEps) ? (yh - yv) / (yh * (1.0f - yh)) * inv_n : 0.0f;
    }
    __shared__ double red[kBceThreads / 32];
    const double v = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kBceThreads / 32; ++w) s += red[w];
        partials[blockIdx.x] = s;
    }
}

__global__ void k_bce_final(double* partials, int nblk, int64_t n) {
    __shared__ double red[32];
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partials[b];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        partials[nblk] = t / (double)n;
    }
}

// ------------------------------------------------------------------ Eq. 10
// Scratch (doubles): [0, nblk) BCE block partials, [nblk, 2 nblk) pooled-MSE block
// partials, [2 nblk] the loss, then 4 ints: the crop's row / column bounds.
constexpr int kEqThreads = 256;

__device__ __forceinline__ int* eq10_box(double* scratch, int nblk) {
    return reinterpret_cast<int*>(scratch + 2 * nblk + 1);
}

__global__ void k_eq10_init(double* scratch, int nblk, int H, int W) {
    int* box = eq10_box(scratch, nblk);
    box[0] = H;   // first row with a non-zero prediction or target
    box[1] = -1;  // last such row
    box[2] = W;
    box[3] = -1;
}

// crop of the BCE term: bounding box of the union of the non-zero entries
__global__ void __launch_bounds__(kEqThreads) k_eq10_box(const float* __restrict__ yhat, const float* __restrict__ y,
                                                         int H, int W, double* scratch, int nblk) {
    int r0 = H, r1 = -1, c0 = W, c1 = -1;
    const int64_t n = (int64_t)H * W;
    for (int64_t i = (int64_t)blockIdx.x * kEqThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kEqThreads) {
        if (yhat[i] != 0.0f || y[i] != 0.0f) {
            const int r = (int)(i / W), c = (int)(i % W);
            r0 = min(r0, r); r1 = max(r1, r); c0 = min(c0, c); c1 = max(c1, c);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        r0 = min(r0, __shfl_down_sync(0xffffffffu, r0, o));
        r1 = max(r1, __shfl_down_sync(0xffffffffu, r1, o));
        c0 = min(c0, __shfl_down_sync(0xffffffffu, c0, o));
        c1 = max(c1, __shfl_down_sync(0xffffffffu, c1, o));
    }
    if ((threadIdx.x & 31) == 0 && r1 >= 0) {
        int* box = eq10_box(scratch, nblk);
        atomicMin(box + 0, r0); atomicMax(box + 1, r1); atomicMin(box + 2, c0); atomicMax(box + 3, c1);
    }
}

// BCE with logits over the crop; dL/dyhat = (sigmoid(x) - y) / N there, 0 elsewhere
__global__ void __launch_bounds__(kEqThreads) k_eq10_bce(const float* __restrict__ yhat, const float* __restrict__ y,
                                                         int H, int W, float* __restrict__ g, double* scratch,
                                                         int nblk) {
    const int* box = eq10_box(scratch, nblk);
    const int r0 = box[0], r1 = box[1], c0 = box[2], c1 = box[3];
    const bool any = r1 >= 0;
    const int64_t N = any ? (int64_t)(r1 - r0 + 1) * (c1 - c0 + 1) : 1;
    const float inv_n = (float)(1.0 / (double)N);
    double acc = 0.0;
    const int64_t n = (int64_t)H * W;
    for (int64_t i = (int64_t)blockIdx.x * kEqThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kEqThreads) {
        const int r = (int)(i / W), c = (int)(i % W);
        float gi = 0.0f;
        if (any && r >= r0 && r <= r1 && c >= c0 && c <= c1) {
            const float x = yhat[i], t = y[i];
            // -[t log s(x) + (1 - t) log(1 - s(x))] = max(x, 0) - t x + log(1 + exp(-|x|))
            acc += (double)(fmaxf(x, 0.0f) - t * x + log1pf(expf(-fabsf(x))));
            const float sg = 1.0f / (1.0f + expf(-x));
            gi = (sg - t) * inv_n;
        }
        if (g) g[i] = gi;
    }
    __shared__ double red[kEqThreads / 32];
    const double v = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kEqThreads / 32; ++w) t += red[w];
        scratch[blockIdx.x] = t;
    }
}

// mean squared difference of the 4 x 4, stride-4 average pools (windows inside the map)
__global__ void __launch_bounds__(kEqThreads) k_eq10_pool(const float* __restrict__ yhat, const float* __restrict__ y,
                                                          int H, int W, float* __restrict__ g, double* scratch,
                                                          int nblk) {
    const int Hp = H / 4, Wp = W / 4;
    const int64_t np = (int64_t)Hp * Wp;
    const float scale = np ? (float)(2.0 / ((double)np * 16.0)) : 0.0f;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kEqThreads + threadIdx.x; i < np; i += (int64_t)gridDim.x * kEqThreads) {
        const int pr = (int)(i / Wp), pc = (int)(i % Wp);
        float sx = 0.0f, sy = 0.0f;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int64_t j = (int64_t)(4 * pr + a) * W + 4 * pc + b;
                sx += yhat[j];
                sy += y[j];
            }
        const float diff = (sx - sy) * (1.0f / 16.0f);
        acc += (double)diff * (double)diff;
        if (g) {
            const float gd = scale * diff;
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) g[(int64_t)(4 * pr + a) * W + 4 * pc + b] += gd;
        }
    }
    __shared__ double red[kEqThreads / 32];
    const double v = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kEqThreads / 32; ++w) t += red[w];
        scratch[nblk + blockIdx.x] = t;
    }
}

// loss = (sum of BCE partials) / N + (sum of pooled partials) / N_pool, fixed order
__global__ void k_eq10_final(double* scratch, int nblk, int H, int W) {
    __shared__ double red[2][32];
    double s0 = 0.0, s1 = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        s0 += scratch[b];
        s1 += scratch[nblk + b];
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = s0;
        red[1][threadIdx.x >> 5] = s1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t0 += red[0][w];
            t1 += red[1][w];
        }
        const int* box = eq10_box(scratch, nblk);
        const double N = box[1] >= 0 ? (double)(box[1] - box[0] + 1) * (double)(box[3] - box[2] + 1) : 1.0;
        const double np = (double)(H / 4) * (double)(W / 4);
        scratch[2 * nblk] = (box[1] >= 0 ? t0 / N : 0.0) + (np > 0 ? t1 / np : 0.0);
    }
}

// ------------------------------------------------------- ensemble metrics
__device__ __forceinline__ bool affected(uint8_t s) { return s == 2 || s == 3; }

// probability of arrival: the fraction of realisations in which the cell burned or burns
__global__ void k_arrival(const uint8_t* __restrict__ S, int R, int64_t HW, float* __restrict__ P) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < HW; j += (int64_t)gridDim.x * blockDim.x) {
        int n = 0;
        for (int r = 0; r < R; ++r) n += affected(S[(int64_t)r * HW + j]);
        P[j] = (float)n / (float)R;  // correctly rounded quotient of the count
    }
}

// integer counts: out[0] += |affected(A) and affected(B)|, out[1] += |either|; or, with
// B == nullptr, out[r] += affected cells of realisation r (blockIdx.y = r)
__global__ void k_count(const uint8_t* __restrict__ A, const uint8_t* __restrict__ B, int64_t n,
                        unsigned long long* __restrict__ out) {
    unsigned long long c0 = 0, c1 = 0;
    const uint8_t* a = A + (B ? 0 : (int64_t)blockIdx.y * n);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const bool x = affected(a[j]);
        if (B) {
            const bool y = affected(B[j]);
            c0 += (x && y);
            c1 += (x || y);
        } else {
            c0 += x;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c0 += __shfl_down_sync(0xffffffffu, c0, o);
        c1 += __shfl_down_sync(0xffffffffu, c1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (B) {
            if (c0) atomicAdd(out + 0, c0);
            if (c1) atomicAdd(out + 1, c1);
        } else if (c0) {
            atomicAdd(out + blockIdx.y, c0);
        }
    }
}

}  // namespace

void launch_arrival(const uint8_t* S, int R, int64_t HW, float* P, cudaStream_t s) {
    const int blocks = (int)std::min<int64_t>(std::max<int64_t>((HW + 255) / 256, 1), 152 * 8);
    k_arrival<<<blocks, 256, 0, s>>>(S, R, HW, P);
}

// Eq. 12 from two series of affected counts: out += sum over t of |a[t] - b[t]| (one block)
__global__ void __launch_bounds__(256) k_l1(const unsigned long long* __restrict__ a,
                                            const unsigned long long* __restrict__ b, int T,
                                            unsigned long long* __restrict__ out) {
    __shared__ unsigned long long sw[8];
    unsigned long long v = 0ull;
    for (int t = threadIdx.x; t < T; t += blockDim.x) v += a[t] > b[t] ? a[t] - b[t] : b[t] - a[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0ull;
        for (int w = 0; w < 8; ++w) t += sw[w];
        *out = t;
    }
}

void launch_l1(const unsigned long long* a, const unsigned long long* b, int T, unsigned long long* out,
               cudaStream_t s) {
    k_l1<<<1, 256, 0, s>>>(a, b, T, out);
}

void launch_count(const uint8_t* A, const uint8_t* B, int64_t n, int R, unsigned long long* out, cudaStream_t s) {
    const int blocks = (int)std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 152 * 4);
    k_count<<<dim3(blocks, B ? 1 : R), 256, 0, s>>>(A, B, n, out);
}

int eq10_blocks(int H, int W) {
    const int64_t n = (int64_t)H * W;
    return (int)std::min<int64_t>(std::max<int64_t>((n + kEqThreads - 1) / kEqThreads, 1), 152 * 8);
}

size_t eq10_scratch_bytes(int H, int W) { return (2 * (size_t)eq10_blocks(H, W) + 1 + 2) * sizeof(double); }

const double* eq10_result(const double* scratch, int nblk) { return scratch + 2 * nblk; }

void launch_eq10(const float* yhat, const float* y, int H, int W, float* g, double* scratch, int nblk,
                 cudaStream_t s) {
    k_eq10_init<<<1, 1, 0, s>>>(scratch, nblk, H, W);
    k_eq10_box<<<nblk, kEqThreads, 0, s>>>(yhat, y, H, W, scratch, nblk);
    k_eq10_bce<<<nblk, kEqThreads, 0, s>>>(yhat, y, H, W, g, scratch, nblk);
    k_eq10_pool<<<nblk, kEqThreads, 0, s>>>(yhat, y, H, W, g, scratch, nblk);
    k_eq10_final<<<1, 1024, 0, s>>>(scratch, nblk, H, W);
}

void launch_validate_fields(const float* x, size_t n, float lo, int bit, int* flags, cudaStream_t s) {
    unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 8);
    k_validate_fields<<<blocks ? blocks : 1, 256, 0, s>>>(x, n, lo, bit, flags);
}

void launch_validate_states(const uint8_t* S, size_t n, int* flags, cudaStream_t s) {
    unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 8);
    k_validate_states<<<blocks ? blocks : 1, 256, 0, s>>>(S, n, flags);
}

void launch_diff_init(const uint8_t* S, int H, int W, int pitch, float* ab, uint8_t* burn, cudaStream_t s) {
    const size_t n = (size_t)H * W;
    k_diff_init<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(S, H, W, pitch, ab, burn);
}

void launch_state_counts(const uint8_t* S, int R, int H, int W, int pitch, unsigned long long* counts,
                         cudaStream_t s) {
    const size_t n = (size_t)R * H * W;
    const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 4096);
    k_state_counts<<<blocks, 256, 0, s>>>(S, R, H, W, pitch, counts);
}

void launch_diff_sums(const float* ab, const uint8_t* burn, int H, int W, int pitch, unsigned long long* nburn,
                      double* sums, cudaStream_t s) {
    const size_t n = (size_t)H * W;
    const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 4096);
    k_diff_sums<<<blocks, 256, 0, s>>>(ab, burn, H, W, pitch, nburn, sums);
}

void launch_diff_pack(const float* dense, int H, int W, int pitch, float* ab, cudaStream_t s) {
    const size_t n = (size_t)H * W;
    k_diff_pack<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dense, H, W, pitch, ab);
}

void launch_diff_unpack(const float* ab, int H, int W, int pitch, float* dense, cudaStream_t s) {
    const size_t n = (size_t)H * W;
    k_diff_unpack<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ab, H, W, pitch, dense);
}

int bce_blocks(int64_t n) {
    int64_t b = (n + kBceThreads - 1) / kBceThreads;
    return (int)std::min<int64_t>(std::max<int64_t>(b, 1), 152 * 8);
}

void launch_bce(const float* a, const float* y, int64_t n, float* g, double* partials, int nblk, cudaStream_t s) {
    k_bce<<<nblk, kBceThreads, 0, s>>>(a, y, n, g, partials);
    k_bce_final<<<1, 1024, 0, s>>>(partials, nblk, n);
}

}  // namespace pf
