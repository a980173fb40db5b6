// pf_loss_bce_noalloc: the binary cross-entropy loss and gradient of pf_loss_bce with
// its reduction scratch in a statically allocated device array instead of memory the
// library allocates on first use. For callers that may not allocate device memory.
#include <cstdio>
#include <mutex>

#include "common.cuh"
#include "pfire.h"

namespace pf {
void launch_bce(const float* a, const float* y, int64_t n, float* g, double* partials, int nblk, cudaStream_t s);
void set_context_free_error(const char* msg);  // read back by pf_last_error(NULL)
}

namespace {

// One FP64 partial sum per block of the first reduction pass plus the final loss.
// Each block covers 4096 elements (256 threads x 16), so the array bounds the problem
// size: n <= PF_NOALLOC_BCE_MAX_N = 16384 * 4096 = 67,108,864 (an 8192 x 8192 map).
constexpr int kMaxBlocks = 16384;
constexpr int64_t kPerBlock = 4096;
static_assert((int64_t)kMaxBlocks * kPerBlock == PF_NOALLOC_BCE_MAX_N, "scratch size and the stated limit differ");

static __device__ __align__(256) double g_bce_scratch[kMaxBlocks + 1];

// Host-side copies of the array's device address, one per device, each with the id of
// the context it was looked up in. The symbol itself is only a host-side stand-in; the
// address comes from cudaGetSymbolAddress with the device current. A context that was
// destroyed and re-created (cudaDeviceReset, or a primary context released and
// retained again) has a new id, and the address is looked up again in it.
constexpr int kMaxDevices = 64;
struct ScratchSlot {
    double* addr;
    unsigned long long ctx_id;
};
ScratchSlot g_scratch[kMaxDevices] = {};
std::mutex g_setup_mutex;

// cuCtxGetCurrent / cuCtxGetId through the runtime's driver entry points (the library
// does not link the driver library itself); false if either is unavailable.
bool current_context_id(unsigned long long* id) {
    using GetCur = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCur get_cur = nullptr;
    static GetId get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<GetCur>(p);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(p);
        cudaGetLastError();
    }
    CUcontext c = nullptr;
    if (!get_cur || !get_id || get_cur(&c) != CUDA_SUCCESS || !c) return false;
    return get_id(c, id) == CUDA_SUCCESS;
}

int set_err(int code, const char* msg, const char* detail = nullptr) {
    char buf[256];
    snprintf(buf, sizeof buf, "pf_loss_bce_noalloc: %s%s%s", msg, detail ? ": " : "", detail ? detail : "");
    pf::set_context_free_error(buf);
    return code;
}

}  // namespace

extern "C" {

int pf_loss_bce_noalloc(const float* a, const float* y, int64_t n, float* dL_da, double* loss, void* cuda_stream) {
    if (!a || !y) return set_err(PF_EINVAL, "a or y is NULL");
    if (n <= 0) return set_err(PF_EINVAL, "n must be >= 1");
    if (n > PF_NOALLOC_BCE_MAX_N)
        return set_err(PF_EINVAL, "n exceeds the 67108864-element limit of the static scratch (use pf_loss_bce)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(PF_ECUDA, "cudaGetDevice failed", cudaGetErrorString(e));
    }
    if (dev < 0 || dev >= kMaxDevices) return set_err(PF_EINVAL, "device ordinal beyond the supported 64");
    double* scratch;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        unsigned long long id = 0;
        // without a context id the address is looked up on every call (a host-side query)
        const bool have_id = current_context_id(&id);
        if (!g_scratch[dev].addr || !have_id || g_scratch[dev].ctx_id != id) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_bce_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                g_scratch[dev].addr = nullptr;
                return set_err(PF_ECUDA, "cudaGetSymbolAddress failed", cudaGetErrorString(e));
            }
            if (!have_id) current_context_id(&id);  // the lookup may have created the context
            g_scratch[dev].addr = static_cast<double*>(p);
            g_scratch[dev].ctx_id = id;
        }
        scratch = g_scratch[dev].addr;
    }
    const int nblk = (int)((n + kPerBlock - 1) / kPerBlock);
    if (nblk > kMaxBlocks) return set_err(PF_EINVAL, "scratch too small for n");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // every call overwrites the nblk + 1 entries it reads; nothing needs clearing
    pf::launch_bce(a, y, n, dL_da, scratch, nblk, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(PF_ECUDA, "launch failed", cudaGetErrorString(e));
    if (loss) {
        double h = 0.0;
        e = cudaMemcpyAsync(&h, scratch + nblk, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_err(PF_ECUDA, "reading the loss failed", cudaGetErrorString(e));
        }
        *loss = h;
    }
    return PF_OK;
}

}  // extern "C"
