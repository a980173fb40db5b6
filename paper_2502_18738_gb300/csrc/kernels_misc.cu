// Small helper kernels: input validation, continuous-state initialisation, and the
// binary cross-entropy loss of a burn-probability map.
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
    const float a = dense[idx];
    ab[j] = a_encode(a, 1.0f - a);
    ab[(size_t)H * pitch + j] = dense[HW + idx];
}

__global__ void k_diff_unpack(const float* __restrict__ ab, int H, int W, int pitch, float* __restrict__ dense) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t HW = (size_t)H * W;
    if (idx >= HW) return;
    const int r = (int)(idx / W), c = (int)(idx % W);
    const size_t j = (size_t)r * pitch + c;
    float a, ua;
    a_decode(ab[j], a, ua);
    dense[idx] = a;
    dense[HW + idx] = ab[(size_t)H * pitch + j];
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

}  // namespace

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
