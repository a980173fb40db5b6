// libpfire C ABI: context, buffers, wind epochs, checkpointed reverse sweep, dispatch.
#include <cudaTypedefs.h>
#include <sys/stat.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "common.cuh"
#include "pfire.h"
#include "tma.cuh"

namespace pf {
// small helper kernels (kernels_misc.cu)
void launch_validate_fields(const float* x, size_t n, float lo, int bit, int* flags, cudaStream_t s);
void launch_validate_states(const uint8_t* S, size_t n, int* flags, cudaStream_t s);
void launch_diff_init(const uint8_t* S, int H, int W, int pitch, float* ab, uint8_t* burn, cudaStream_t s);
void launch_state_counts(const uint8_t* S, int R, int H, int W, int pitch, unsigned long long* counts, cudaStream_t s);
void launch_diff_sums(const float* ab, const uint8_t* burn, int H, int W, int pitch, unsigned long long* nburn,
                      double* sums, cudaStream_t s);
void launch_bce(const float* a, const float* y, int64_t n, float* g, double* partials, int nblk, cudaStream_t s);
void launch_arrival(const uint8_t* S, int R, int64_t HW, float* P, cudaStream_t s);
void launch_count(const uint8_t* A, const uint8_t* B, int64_t n, int R, unsigned long long* out, cudaStream_t s);
void launch_l1(const unsigned long long* a, const unsigned long long* b, int T, unsigned long long* out,
               cudaStream_t s);
int eq10_blocks(int H, int W);
size_t eq10_scratch_bytes(int H, int W);
const double* eq10_result(const double* scratch, int nblk);
void launch_eq10(const float* yhat, const float* y, int H, int W, float* g, double* scratch, int nblk, cudaStream_t s);
int bce_blocks(int64_t n);
}  // namespace pf

using namespace pf;

namespace {

thread_local std::string g_last_error = "no error";

enum Kind {
    K_PREP, K_DSTEP, K_DBLK, K_FSTEP, K_FBLK, K_ADJ, K_ABLK, K_PADJ, K_RED, K_MISC, K_ATILES, K_FTILES, K_DCA,
    K_STILES, K_AFRZ, K_TUNPACK, K_NKINDS
};
const char* kKindNames[K_NKINDS] = {"prep",         "discrete_step",    "discrete_blocked",
                                    "diff_step",    "diff_blocked",     "adjoint_step",
                                    "adjoint_blocked", "prep_adjoint",  "reduce_fp64",
                                    "misc",         "adjoint_tiles",    "diff_tiles",
                                    "dca_step",     "segment_tiles",    "adjoint_frozen",
                                    "segment_from_tape"};

struct Epoch {
    int from;
    float* V;   // dense H*W or nullptr (calm)
    float* th;  // dense H*W or nullptr
    cudaEvent_t ready = nullptr;  // upload of pf_set_wind_async done (on the copy stream)
};

struct ProfRec {
    int kind;
    cudaEvent_t e0, e1;
};

// Host-side allocation-failure injector: PF_FAULT_ALLOC=n makes the n-th device
// allocation of the process fail with PF_ENOMEM (n >= 1).
long g_alloc_count = 0;
long fault_alloc_at() {
    static long at = -2;
    if (at == -2) {
        const char* s = getenv("PF_FAULT_ALLOC");
        at = s ? atol(s) : -1;
    }
    return at;
}

// The TMA kernels' test hook from the environment: PF_TMA_TEST_WITHHOLD=1 makes them arm
// their barriers without issuing the copies, PF_TMA_SPIN_LIMIT=n bounds each wait to n
// polls (default kSpinLimit). Read at each call that launches them, so a test can turn
// it on and off between calls.
pf::TmaHook read_tma_hook() {
    pf::TmaHook h{pf::kSpinLimit, 0};
    if (const char* w = getenv("PF_TMA_TEST_WITHHOLD")) h.withhold = atoi(w) != 0;
    if (const char* l = getenv("PF_TMA_SPIN_LIMIT")) {
        const long v = atol(l);
        if (v > 0) h.spin = (uint32_t)v;
    }
    return h;
}

}  // namespace

namespace pf {
void set_context_free_error(const char* msg) { g_last_error = msg; }
}  // namespace pf

struct pf_ctx {
    int H = 0, W = 0, P = 0, form = 0, R = 1;
    uint64_t seed = 0;
    cudaStream_t st = nullptr;
    float p_h = 0.58f, c1 = 0.045f, c2 = 0.131f, a = 0.078f, pc = 0.3f, l = 30.0f;
    float *E = nullptr, *pveg = nullptr, *pden = nullptr;
    std::vector<Epoch> winds;
    std::vector<float*> wind_pool;  // H*W buffers of dropped wind epochs, reused
    cudaStream_t cst = nullptr;     // copy stream of pf_set_wind_async (created on first use)
    // q cache
    float* q = nullptr;      // q of the current wind epoch (q_own or one of qcache)
    float* q_own = nullptr;  // the context's own q buffer
    // per-epoch q kept from a taped forward for its adjoint (differentiable form, when
    // the epochs fit in 30% of the free memory), with the version each was made at
    std::vector<float*> qcache;
    std::vector<long> qcache_ver;
    // differentiable form: a q computed under a reach mask is valid for the steps before
    // q_until (qcache_until[e] for the cached ones) of the trajectory it was made on
    std::vector<int> qcache_until;
    int q_until = 0x7fffffff;
    uint8_t* qreach = nullptr;  // reach mask and its scratch (2 x prep_reach_bytes)
    // a taped forward without the q cache: the union of the reach masks each epoch's q
    // was computed under (qmasks[e * prep_reach_bytes ..]), so that the adjoint recomputes
    // q in the same blocks; qmask_state[e] 0 none, 1 masked, 2 every cell
    uint8_t* qmasks = nullptr;
    int qmasks_cap = 0;  // epochs
    std::vector<int> qmask_state;
    bool qcache_on = false;
    long q_key_epoch = -1;
    long q_key_version = -1;
    long version = 0;  // bumped whenever params / env / wind / mask change
    // state
    int step = 0;
    uint8_t* S[2] = {nullptr, nullptr};  // discrete [R][H][P]
    int scur = 0;
    // the paper's accumulator path (discrete form): caller's accumulator [R][H][W], the
    // initial state of the recorded trajectory and the context version it was run with
    float* acc = nullptr;
    float* slope = nullptr;  // H x W x 3 x 3 slope input (degrees), replaces E when set
    uint8_t* dca_S0 = nullptr;
    uint8_t* dca_S[2] = {nullptr, nullptr};
    bool dca_valid = false;
    long long dca_version = -1;
    float* work[2] = {nullptr, nullptr};  // diff [2][H][P]
    float* cur_ab = nullptr;              // where the current diff state lives
    uint8_t* burn = nullptr;              // diff burnable mask, dense H*W
    // tape (diff)
    bool tape_valid = false;
    int tape_start = 0;
    int K = 1;
    std::vector<std::pair<int, int>> ckpts;  // (step, arena slot)
    float* arena = nullptr;                  // consecutive saved states, slot i at arena + i * state
    int arena_cap = 0, arena_used = 0;
    float t_p_h = 0, t_c1 = 0, t_c2 = 0, t_a = 0, t_pc = 0, t_l = 0;
    long t_version = -1;
    // adjoint
    float* lam[2] = {nullptr, nullptr};   // scaled adjoint mu (lambda = mu 2^sigma)
    uint8_t* sig[2] = {nullptr, nullptr};  // its per-cell exponents sigma
    float* Gq = nullptr;
    double* partials = nullptr;
    double* gacc = nullptr;
    // misc
    int* dflags = nullptr;  // [0] device error word, [1] validation, [3] async wind validation
    int* hflags = nullptr;  // pinned mirror
    unsigned long long* dskip = nullptr;  // per kernel kind: cell-steps of skipped quiescent tiles
    // discrete near-tie counters ([0] ignition, [1] continue, since the last pf_forward)
    // and pf_stats scratch ([2..5] state counts, [6..7] FP64 sums of a and b)
    unsigned long long* dties = nullptr;
    // test hook of the TMA kernels, read from the environment at each forward / backward
    // (PF_TMA_TEST_WITHHOLD, PF_TMA_SPIN_LIMIT)
    TmaHook hook{kSpinLimit, 0};
    int* tile_list = nullptr;             // tiles of one blocked-adjoint launch (counts: dflags[8], [10]; work: [9], [11])
    uint8_t* gqdirty = nullptr;           // per adjoint tile: may hold nonzero dL/dq this epoch
    // tile activity of the blocked forward (b > 0 in a tile's interior), carried along a
    // chain of launches: act ping-pong, quiescent-last-launch flags, live list (count: dflags[12])
    uint8_t* fact[2] = {nullptr, nullptr};
    uint8_t* fqrun = nullptr;  // per tile: quiescent streak along the chain (k_fwd_tiles)
    int* flist = nullptr;
    const float* fl_state = nullptr;    // the state fact[fl_par] describes (nullptr: none)
    int fl_launch = 0;                  // launches of the chain so far
    const uint8_t* fl_seed = nullptr;   // flags recorded for the next chain's first state (or none)
    int fl_seed_halo = 0;
    // per arena slot: the tile flags the blocked forward recorded for the checkpoint it
    // wrote there (ckact + slot * tiles), with their halo (0: none)
    uint8_t* ckact = nullptr;
    int ckact_cap = 0;
    std::vector<int> ckact_halo;
    // per arena slot and forward tile: whether the slot's tile may hold nonzeros, valid
    // for the tile geometry (halo) ckdirty_halo[slot] (0: unknown, every tile is written)
    uint8_t* ckdirty = nullptr;
    int ckdirty_cap = 0;
    std::vector<int> ckdirty_halo;
    int fl_in_at[2] = {-1, -1};         // launch whose input work[x] last was (-1: none)
    int fl_par = 0;
    int fl_halo = 0;
    // the tile activity at the end of every launch of a taped (K = 1) forward or of a
    // segment's recompute, for the adjoint's tile lists: actrec_end[i] is the step whose
    // state slot i describes; adeadcnt counts the adjoint's quiescent launches per tile
    uint8_t* actrec = nullptr;
    int actrec_cap = 0;
    std::vector<int> actrec_end;
    bool actrec_on = false;
    uint8_t* adeadcnt = nullptr;
    CUtensorMap tmapS[2];
    bool tmap_ok = false;
    CUtensorMap tmapQ;       // q planes (pitch, H, 8), box of the blocked diff kernel
    bool tmapQ_ok = false;
    int nsm = 152;
    float* seg_buf = nullptr;  // K-1 contiguous states (segment recompute)
    int seg_cap = 0;
    uint32_t* seg_rng = nullptr;  // per forward tile: slots [lo, hi) of seg_buf (from slot 1) where its interior may be nonzero
    const float* seg_slot0 = nullptr;  // the segment's first state (its checkpoint; slot 0 of seg_buf is unused)
    int seg_halo = 0;              // tile geometry seg_dirty refers to
    // tile tape of a checkpointed taped forward (TileTape in common.cuh): the live tiles'
    // states of every blocked launch, so that the backward copies a segment's states
    // instead of recomputing them; records (t0, n) of this tape's launches, their device
    // records {base, n, count, ok} and lists
    float* ttape = nullptr;
    unsigned long long ttape_cap = 0;      // blocks
    size_t ttape_blk = 0;                  // bytes a block
    unsigned long long* ttape_used = nullptr;
    unsigned long long* ttape_meta = nullptr;
    int* ttape_lists = nullptr;
    int* ttape_inv = nullptr;
    int ttape_rec_cap = 0;
    std::vector<std::pair<int, int>> ttape_rec;
    std::vector<unsigned long long> ttape_meta_h;  // host copy of the records (backward)
    bool ttape_on = false;
    // the last tape ran out of blocks (some launches were left out and recomputed)
    bool ttape_short = false;
    // blocks the last taped forward asked for (recorded or not), at block size ttape_need_blk
    unsigned long long ttape_need = 0;
    size_t ttape_need_blk = 0;
    int TH = 64, KH = 16;
    // Philox counter words 3 and 1 (base) of the discrete draws: 0 for contexts made by
    // pf_create; a batch job run through a context of its own uses its fire_id and run
    uint32_t fire_id = 0, run0 = 0;
    // device memory from this stream-ordered pool (allocations and frees ordered on st,
    // no device-wide synchronisation), or from cudaMalloc when null
    cudaMemPool_t pool = nullptr;
    pf_tuning tun{0, 0, 0, 0, 0, 0, 0};
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> ev_pool;
    long long launches[K_NKINDS] = {0};
    long long cell_steps[K_NKINDS] = {0};
    double prof_ms[K_NKINDS] = {0};
    std::vector<void*> allocs;
    long long n_allocs = 0, n_frees = 0;  // device allocations and frees made so far
    std::string err = "no error";
};

namespace {

int fail(pf_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    g_last_error = buf;
    return code;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(ctx, PF_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));       \
    } while (0)

// the pool of the contexts pf_create makes on this thread (the batch's direct jobs)
thread_local cudaMemPool_t g_ctx_pool = nullptr;

int dalloc(pf_ctx* ctx, void** p, size_t bytes) {
    *p = nullptr;
    ++g_alloc_count;
    const long at = fault_alloc_at();
    if (at > 0 && g_alloc_count == at)
        return fail(ctx, PF_ENOMEM, "injected allocation failure (PF_FAULT_ALLOC=%ld)", at);
    cudaError_t e = ctx->pool ? cudaMallocFromPoolAsync(p, bytes ? bytes : 16, ctx->pool, ctx->st)
                              : cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(ctx, PF_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    ctx->allocs.push_back(*p);
    ++ctx->n_allocs;
    return PF_OK;
}

void dfree(pf_ctx* ctx, void* p) {
    if (!p) return;
    ++ctx->n_frees;
    auto it = std::find(ctx->allocs.begin(), ctx->allocs.end(), p);
    if (it != ctx->allocs.end()) ctx->allocs.erase(it);
    if (ctx->pool) cudaFreeAsync(p, ctx->st);
    else cudaFree(p);
}

size_t plane_elems(const pf_ctx* c) { return (size_t)c->H * c->P; }
size_t diff_state_bytes(const pf_ctx* c) { return 2 * plane_elems(c) * sizeof(float); }

// ------------------------------------------------------------- profiling
struct LaunchScope {
    pf_ctx* c;
    int kind;
    cudaEvent_t e1 = nullptr;
    // steps: automaton steps the launch advances (or reverses) every cell by
    LaunchScope(pf_ctx* c_, int k, int steps = 1) : c(c_), kind(k) {
        c->launches[k] += 1;
        if (k != K_MISC && k != K_PREP && k != K_PADJ && k != K_RED && k != K_ATILES && k != K_FTILES &&
            k != K_DCA && k != K_STILES && k != K_AFRZ && k != K_TUNPACK)
            c->cell_steps[k] += (long long)steps * c->H * c->W * (k == K_DSTEP || k == K_DBLK ? c->R : 1);
        if (!c->tun.profile) return;
        cudaEvent_t e0 = take();
        e1 = take();
        cudaEventRecord(e0, c->st);
        c->prof.push_back({k, e0, e1});
    }
    ~LaunchScope() {
        if (e1) cudaEventRecord(e1, c->st);
    }
    cudaEvent_t take() {
        if (!c->ev_pool.empty()) {
            cudaEvent_t e = c->ev_pool.back();
            c->ev_pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
};

void prof_collect(pf_ctx* c) {
    for (auto& r : c->prof) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) c->prof_ms[r.kind] += ms;
        c->ev_pool.push_back(r.e0);
        c->ev_pool.push_back(r.e1);
    }
    c->prof.clear();
    cudaGetLastError();
}

int check_launch(pf_ctx* ctx, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, PF_ECUDA, "%s launch failed: %s", what, cudaGetErrorString(e));
    return PF_OK;
}

// ------------------------------------------------------------- TMA maps
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    }
    return fn;
}

bool encode_state_map(pf_ctx* c, CUtensorMap* m, uint8_t* base) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)c->P, (cuuint64_t)c->H, (cuuint64_t)c->R};
    cuuint64_t strides[2] = {(cuuint64_t)c->P, (cuuint64_t)c->P * c->H};
    cuuint32_t box[3] = {160u, (cuuint32_t)(c->TH + 2 * c->KH), 1u};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, base, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool encode_f32_3d(CUtensorMap* m, const float* base, int P, int H, int planes, int box_c, int box_r, int box_p) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)P, (cuuint64_t)H, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)P * 4, (cuuint64_t)P * H * 4};
    cuuint32_t box[3] = {(cuuint32_t)box_c, (cuuint32_t)box_r, (cuuint32_t)box_p};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// ------------------------------------------------------------- q cache
int epoch_of(const pf_ctx* c, int t) {
    int e = 0;
    for (size_t i = 0; i < c->winds.size(); ++i)
        if (t >= c->winds[i].from) e = (int)i;
    return e;
}

int next_epoch_start(const pf_ctx* c, int t) {
    for (auto& w : c->winds)
        if (w.from > t) return w.from;
    return 0x7fffffff;
}

// Arguments of the prep kernels for wind epoch e. The caller launches on c->st next, so
// an epoch still being uploaded by pf_set_wind_async is waited for here (a wait of the
// stream on the upload's event; the host does not block).
PrepArgs prep_args(pf_ctx* c, int e, bool use_tape_params) {
    if (c->winds[e].ready) cudaStreamWaitEvent(c->st, c->winds[e].ready, 0);  // an error is caught by check_launch
    PrepArgs g{};
    g.H = c->H; g.W = c->W; g.pitch = c->P;
    g.E = c->E; g.pveg = c->pveg; g.pden = c->pden;
    g.V = c->winds[e].V; g.th = c->winds[e].th;
    g.burnable = (c->form == PF_DIFF) ? c->burn : nullptr;
    g.slope = c->slope;
    if (use_tape_params) {
        g.p_h = c->t_p_h; g.c1 = c->t_c1; g.c2 = c->t_c2; g.a = c->t_a; g.l = c->t_l;
    } else {
        g.p_h = c->p_h; g.c1 = c->c1; g.c2 = c->c2; g.a = c->a; g.l = c->l;
    }
    prep_derive(g);
    return g;
}

// Point the kernels at another q buffer (the blocked diff kernels read q through a
// tensor map, re-encoded here).
int use_q_buffer(pf_ctx* ctx, float* buf) {
    if (ctx->q == buf) return PF_OK;
    ctx->q = buf;
    if (ctx->form == PF_DIFF && ctx->tmapQ_ok &&
        !encode_f32_3d(&ctx->tmapQ, buf, ctx->P, ctx->H, 8, diff_blocked_box_cols(), diff_blocked_box_rows(), 8))
        return fail(ctx, PF_ECUDA, "tensor map encoding of q failed");
    return PF_OK;
}

// Record, for the adjoint of a taped forward that keeps no q cache, which blocks the prep
// of epoch e just computed: the reach mask in ctx->qreach (masked) or every cell.
int qmask_record(pf_ctx* ctx, int e, bool masked) {
    if (!ctx->tape_valid || ctx->qcache_on || ctx->version != ctx->t_version || e < 0) return PF_OK;
    const int ne = (int)ctx->winds.size();
    if (e >= ne) return PF_OK;
    if ((int)ctx->qmask_state.size() < ne) ctx->qmask_state.resize(ne, 0);
    int& st = ctx->qmask_state[e];
    if (!masked || st == 2) {
        st = 2;
        return PF_OK;
    }
    const int nb = prep_reach_bytes(ctx->H, ctx->W);
    if (ctx->qmasks_cap < ne) {
        if (ctx->qmasks) dfree(ctx, ctx->qmasks);
        ctx->qmasks = nullptr;
        ctx->qmasks_cap = 0;
        void* p;
        if (dalloc(ctx, &p, (size_t)nb * ne) != PF_OK) {
            cudaGetLastError();
            st = 2;  // no record: the adjoint computes every cell
            return PF_OK;
        }
        ctx->qmasks = (uint8_t*)p;
        ctx->qmasks_cap = ne;
        for (int k = 0; k < ne; ++k)  // the old records went with the old buffer
            if (ctx->qmask_state[k] == 1 && k != e) ctx->qmask_state[k] = 2;
    }
    uint8_t* m = ctx->qmasks + (size_t)e * nb;
    if (st == 0)
        CK(cudaMemcpyAsync(m, ctx->qreach, (size_t)nb, cudaMemcpyDeviceToDevice, ctx->st));
    else
        launch_reach_or(m, ctx->qreach, nb, ctx->st);
    st = 1;
    return check_launch(ctx, "reach mask record");
}

// q of wind epoch e, valid for the steps before `until` of the current trajectory. In the
// differentiable form a bounded `until` lets prep skip the cells nothing reads before
// then: the region a > 0 grows by at most one cell per step, and every kernel reads q
// only within a few tiles (at most 128 cells) of a cell with a > 0 (the blocked kernels'
// tile regions) or where a burning neighbour multiplies it (elsewhere it multiplies a
// zero). So q is computed only in the 32 x 32 blocks within (until - step) + 160 cells
// of the current a > 0 cells. The other cells keep the buffer's finite values: q buffers
// are zeroed when allocated and only ever receive q values.
int ensure_q(pf_ctx* ctx, int e, int until = 0x7fffffff) {
    int rc;
    const bool masked = ctx->form == PF_DIFF && until != 0x7fffffff && ctx->cur_ab != nullptr;
    if (!masked) until = 0x7fffffff;
    // a taped forward keeps every epoch's q for the adjoint when the cache is on
    const bool cache = ctx->qcache_on && ctx->tape_valid && e < (int)ctx->qcache.size();
    if (cache && ctx->qcache[e] && ctx->qcache_ver[e] == ctx->version && until <= ctx->qcache_until[e]) {
        if ((rc = use_q_buffer(ctx, ctx->qcache[e]))) return rc;
        ctx->q_key_epoch = e;
        ctx->q_key_version = ctx->version;
        ctx->q_until = ctx->qcache_until[e];
        return PF_OK;
    }
    if (cache && !ctx->qcache[e]) {
        void* p;
        if (dalloc(ctx, &p, 8 * plane_elems(ctx) * sizeof(float)) == PF_OK) {
            ctx->qcache[e] = (float*)p;
            CK(cudaMemsetAsync(p, 0, 8 * plane_elems(ctx) * sizeof(float), ctx->st));
        } else {
            cudaGetLastError();
        }
    }
    float* dst = (cache && ctx->qcache[e]) ? ctx->qcache[e] : ctx->q_own;
    if (ctx->q == dst && ctx->q_key_epoch == e && ctx->q_key_version == ctx->version && until <= ctx->q_until)
        return PF_OK;
    if ((rc = use_q_buffer(ctx, dst))) return rc;
    PrepArgs g = prep_args(ctx, e, false);
    {
        LaunchScope ls(ctx, K_PREP);
        if (masked) {
            const int nb = prep_reach_bytes(ctx->H, ctx->W);
            if (!ctx->qreach) {
                void* p;
                if ((rc = dalloc(ctx, &p, 2 * (size_t)nb))) return rc;
                ctx->qreach = (uint8_t*)p;
            }
            const long reach = (long)(until - ctx->step) + 160;
            const int radius = (int)std::min<long>((reach + 31) / 32 + 1, 1L << 20);
            launch_prep_reach(ctx->cur_ab, ctx->H, ctx->W, ctx->P, radius, ctx->qreach + nb, ctx->qreach, ctx->st);
            g.reach = ctx->qreach;
            g.reach_bw = (ctx->W + 31) / 32;
        }
        launch_prep(g, ctx->q, ctx->st);
    }
    rc = check_launch(ctx, "prep");
    if (rc) return rc;
    if ((rc = qmask_record(ctx, e, masked))) return rc;
    if (dst != ctx->q_own) {
        ctx->qcache_ver[e] = ctx->version;
        ctx->qcache_until[e] = until;
    }
    ctx->q_key_epoch = e;
    ctx->q_key_version = ctx->version;
    ctx->q_until = until;
    return PF_OK;
}

int sync_flags(pf_ctx* ctx, int n) {
    CK(cudaMemcpyAsync(ctx->hflags, ctx->dflags, sizeof(int) * n, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return PF_OK;
}

// Synchronises the context's streams and reports what the device recorded since the last
// call: a bounded wait that ran out (PF_ETIMEOUT), else invalid values in a wind epoch
// uploaded by pf_set_wind_async (PF_EINVAL). Both words are cleared once reported.
int device_error(pf_ctx* ctx) {
    if (ctx->cst) CK(cudaStreamSynchronize(ctx->cst));
    int rc = sync_flags(ctx, 4);
    if (rc) return rc;
    if (ctx->hflags[0] != 0) {
        const int code = ctx->hflags[0];
        CK(cudaMemsetAsync(ctx->dflags, 0, sizeof(int), ctx->st));
        return fail(ctx, PF_ETIMEOUT, "a bounded device wait ran out (device code %d)", code);
    }
    if (ctx->hflags[3] != 0) {
        const int bits = ctx->hflags[3];
        CK(cudaMemsetAsync(ctx->dflags + 3, 0, sizeof(int), ctx->st));
        return fail(ctx, PF_EINVAL, "pf_set_wind_async: NaN or infinite values in an uploaded %s",
                    bits == 1 ? "V_w" : bits == 2 ? "theta_w" : "V_w and theta_w");
    }
    return PF_OK;
}

// ------------------------------------------------------------- kernel choice
int choose_kernel(const pf_ctx* c) {
    if (c->tun.kernel == 1) return 1;
    // kernel 2 or automatic: the temporal-blocked kernel when its tensor maps exist
    const bool ok = (c->form == PF_DISCRETE) ? c->tmap_ok : c->tmapQ_ok;
    return ok ? 2 : 1;
}

int blocked_k(const pf_ctx* c) {
    int k = c->tun.k > 0 ? c->tun.k : 8;
    return std::min(k, c->form == PF_DISCRETE ? std::min(c->KH, discrete_blocked_max_k()) : diff_blocked_halo());
}

// One launch of the blocked diff kernel from `in`; out / all_out as in launch_diff_blocked.
// Launches form chains (the output of one is the input of the next) along which the
// tile activity is carried; a chain starts wherever `in` is not the state the activity
// describes (ctx->fl_state, reset by every caller that starts a new sequence).
// keep the activity flags of the state at `end_step` (just produced in fact[fl_par])
int actrec_push(pf_ctx* ctx, int end_step) {
    const size_t nt = (size_t)diff_blocked_tiles(8, ctx->H, ctx->P);
    const int i = (int)ctx->actrec_end.size();
    if (i >= ctx->actrec_cap) {
        const int cap = std::max(16, 2 * ctx->actrec_cap);
        void* p;
        int rc = dalloc(ctx, &p, nt * cap);
        if (rc) return rc;
        if (ctx->actrec) {
            CK(cudaMemcpyAsync(p, ctx->actrec, nt * ctx->actrec_cap, cudaMemcpyDeviceToDevice, ctx->st));
            dfree(ctx, ctx->actrec);
        }
        ctx->actrec = (uint8_t*)p;
        ctx->actrec_cap = cap;
    }
    CK(cudaMemcpyAsync(ctx->actrec + nt * i, ctx->fact[ctx->fl_par], nt, cudaMemcpyDeviceToDevice, ctx->st));
    ctx->actrec_end.push_back(end_step);
    return PF_OK;
}

// Dirty bits of arena slot s for tile geometry `halo` (allocated on first use).
uint8_t* ckpt_dirty_bits(pf_ctx* ctx, int s, int* rc) {
    const size_t nt = (size_t)std::max(diff_blocked_tiles(8, ctx->H, ctx->P), diff_blocked_tiles(4, ctx->H, ctx->P));
    *rc = PF_OK;
    if (ctx->ckdirty_cap < ctx->arena_cap) {
        void* p;
        if ((*rc = dalloc(ctx, &p, nt * (size_t)ctx->arena_cap))) return nullptr;
        if (ctx->ckdirty) dfree(ctx, ctx->ckdirty);
        ctx->ckdirty = (uint8_t*)p;
        ctx->ckdirty_cap = ctx->arena_cap;
        std::fill(ctx->ckdirty_halo.begin(), ctx->ckdirty_halo.end(), 0);
    }
    return ctx->ckdirty + nt * (size_t)s;
}

// A launch of the blocked forward from `in` (n steps). rec >= 0 (a segment recompute):
// the states of the listed tiles come from tile-tape record rec instead of the kernel.
// record (a taped forward with the tile tape on): the listed tiles' states are also
// written into the tape, as a new record.
int diff_blocked_launch(pf_ctx* ctx, const float* in, float pc, int n, float* out, float* all_out,
                        bool seg = false, int end_step = -1, bool frozen = false, const PrepArgs* pa = nullptr,
                        int ckpt_slot = -1, int rec = -1, bool record = false) {
    CUtensorMap tab;
    if (!encode_f32_3d(&tab, in, ctx->P, ctx->H, 2, diff_blocked_box_cols(), diff_blocked_box_rows(), 2))
        return fail(ctx, PF_ECUDA, "tensor map encoding of the state buffer failed");
    const int halo = blocked_k(ctx) <= 4 ? 4 : 8;
    if (ctx->fl_state != in || ctx->fl_halo != halo) {
        {
            LaunchScope ls(ctx, K_FTILES);
            if (ctx->fl_seed && ctx->fl_seed_halo == halo)
                launch_fwd_act_seed(halo, ctx->fl_seed, ctx->H, ctx->P, ctx->fact[ctx->fl_par], ctx->fqrun, ctx->st);
            else
                launch_fwd_act_init(halo, in, ctx->H, ctx->P, ctx->fact[ctx->fl_par], ctx->fqrun, ctx->st);
        }
        ctx->fl_seed = nullptr;
        ctx->fl_halo = halo;
        ctx->fl_launch = 0;
        ctx->fl_in_at[0] = ctx->fl_in_at[1] = -1;
    }
    const size_t stride = 2 * plane_elems(ctx);
    uint8_t* dirty = nullptr;
    bool dirty_unknown = true;
    if (ckpt_slot >= 0) {
        int rc;
        dirty = ckpt_dirty_bits(ctx, ckpt_slot, &rc);
        if (rc) return rc;
        dirty_unknown = ctx->ckdirty_halo[ckpt_slot] != halo;
        ctx->ckdirty_halo[ckpt_slot] = halo;
    }
    // out, if a work buffer, holds the input state of the launch it last was the input of
    // (each launch's output becomes the next one's input, and is complete after it)
    int out_age = 0;
    for (int x = 0; x < 2; ++x)
        if (out && out == ctx->work[x] && ctx->fl_in_at[x] >= 0) out_age = ctx->fl_launch - ctx->fl_in_at[x];
    {
        // the pre-pass of a forward launch, or of one recomputing a segment for the adjoint
        LaunchScope ls(ctx, seg ? K_STILES : K_FTILES);
        if (!launch_fwd_tiles(halo, in, ctx->H, ctx->W, ctx->P, n, ctx->fact[ctx->fl_par], ctx->fact[1 - ctx->fl_par],
                         ctx->fqrun, ctx->flist, ctx->dflags + 12, out, out_age, all_out,
                         stride, seg ? ctx->seg_rng : nullptr, seg ? ctx->seg_slot0 : nullptr,
                         seg ? ctx->seg_buf + stride : nullptr,
                         ctx->seg_cap - 1, seg && frozen && halo == 8, dirty, dirty_unknown,
                         ctx->dskip + (rec >= 0 ? K_TUNPACK : K_FBLK), ctx->dskip + (seg ? K_STILES : K_FTILES),
                         ctx->st))
            return fail(ctx, PF_EINVAL, "segment launch outside the segment buffer");
    }
    if (rec >= 0) {
        LaunchScope ls(ctx, K_TUNPACK);
        const unsigned long long* m = &ctx->ttape_meta_h[4 * (size_t)rec];
        const size_t nt = (size_t)diff_blocked_tiles(halo, ctx->H, ctx->P);
        launch_tape_unpack(halo, ctx->ttape, m[0], (int)m[1], (int)m[2], ctx->ttape_lists + nt * (size_t)rec,
                           ctx->ttape_inv, (int)nt, ctx->flist, ctx->dflags + 12, n, ctx->H, ctx->P, all_out, stride,
                           ctx->fact[1 - ctx->fl_par], ctx->dflags + 14, ctx->nsm, ctx->st);
    } else {
        LaunchScope ls(ctx, K_FBLK, n);
        const TileTape tape{record ? ctx->ttape : nullptr, ctx->ttape_used, ctx->ttape_cap};
        launch_diff_blocked(halo, &tab, &ctx->tmapQ, pa, ctx->H, ctx->W, ctx->P, pc, n, ctx->flist, ctx->dflags + 12, out,
                            all_out, stride, ctx->fact[1 - ctx->fl_par], ctx->dskip + K_FBLK, ctx->nsm, ctx->dflags,
                            ctx->hook, tape, ctx->st);
    }
    if (record) {
        LaunchScope ls(ctx, K_MISC);
        const int L = (int)ctx->ttape_rec.size();
        const int nt = diff_blocked_tiles(halo, ctx->H, ctx->P);
        launch_tape_record(TileTape{ctx->ttape, ctx->ttape_used, ctx->ttape_cap}, ctx->dflags + 12, ctx->flist, n, L,
                           ctx->ttape_meta, ctx->ttape_lists, nt, ctx->st);
        ctx->ttape_rec.push_back({ctx->step, n});
    }
    ctx->fl_par ^= 1;
    ctx->fl_state = out ? out : all_out + (size_t)(n - 1) * stride;
    for (int x = 0; x < 2; ++x)
        if (in == ctx->work[x]) ctx->fl_in_at[x] = ctx->fl_launch;
    ctx->fl_launch++;
    if (ctx->actrec_on && end_step >= 0 && halo == 8) {
        int rc = actrec_push(ctx, end_step);
        if (rc) return rc;
    }
    return check_launch(ctx, "diff blocked");
}

// ------------------------------------------------------------- discrete runs
DiscreteArgs dargs(const pf_ctx* c) {
    DiscreteArgs g;
    g.H = c->H; g.W = c->W; g.pitch = c->P; g.R = c->R;
    g.p_continue = c->pc;
    g.key0 = (uint32_t)c->seed; g.key1 = (uint32_t)(c->seed >> 32);
    g.fire = c->fire_id; g.run0 = c->run0;
    g.acc = c->acc;
    g.acc_r0 = 0; g.acc_r1 = c->H; g.acc_c0 = 0; g.acc_c1 = c->W;
    g.ties = c->dties;
    return g;
}

int run_discrete(pf_ctx* ctx, int T) {
    const DiscreteArgs g = dargs(ctx);
    const int kern = choose_kernel(ctx);
    const bool rcq = ctx->tun.prep == 2;  // q recomputed inside the step kernels
    int t = ctx->step;
    const int end = ctx->step + T;
    int pa_epoch = -1;
    PrepArgs pa{};
    while (t < end) {
        const int e = epoch_of(ctx, t);
        int rc;
        if (rcq) {
            if (e != pa_epoch) pa = prep_args(ctx, e, false);
            pa_epoch = e;
        } else if ((rc = ensure_q(ctx, e))) {
            return rc;
        }
        int n = std::min(end - t, next_epoch_start(ctx, t) - t);
        const int src = ctx->scur, dst = 1 - ctx->scur;
        if (kern == 2) {
            n = std::min(n, blocked_k(ctx));
            LaunchScope ls(ctx, K_DBLK, n);
            launch_discrete_blocked_impl(g, &ctx->tmapS[src], ctx->TH, ctx->KH, ctx->S[dst], ctx->q,
                                         rcq ? &pa : nullptr, (uint32_t)t, n, ctx->dflags, ctx->hook,
                                         ctx->dskip + K_DBLK, ctx->st);
        } else {
            n = 1;
            LaunchScope ls(ctx, K_DSTEP);
            if (rcq)
                launch_discrete_step_rc(g, ctx->S[src], ctx->S[dst], pa, (uint32_t)t, ctx->st);
            else
                launch_discrete_step(g, ctx->S[src], ctx->S[dst], ctx->q, (uint32_t)t, ctx->st);
        }
        rc = check_launch(ctx, "discrete step");
        if (rc) return rc;
        ctx->scur = dst;
        t += n;
    }
    ctx->step = end;
    return PF_OK;
}

// ------------------------------------------------------------- diff runs
float* slot_ptr(const pf_ctx* c, int slot) { return c->arena + (size_t)slot * 2 * plane_elems(c); }

// Make room for `need` slots in the tape arena; a larger arena takes over the used
// slots (and the current-state pointer if it points into them).
int arena_reserve(pf_ctx* ctx, int need) {
    if (need <= ctx->arena_cap) return PF_OK;
    const size_t sb = diff_state_bytes(ctx);
    void* p = nullptr;
    int rc = dalloc(ctx, &p, sb * (size_t)need);
    if (rc) return rc;
    float* old = ctx->arena;
    if (old && ctx->arena_used)
        CK(cudaMemcpyAsync(p, old, sb * (size_t)ctx->arena_used, cudaMemcpyDeviceToDevice, ctx->st));
    if (old && ctx->cur_ab >= old && ctx->cur_ab < old + (size_t)ctx->arena_cap * 2 * plane_elems(ctx))
        ctx->cur_ab = (float*)p + (ctx->cur_ab - old);
    if (old) dfree(ctx, old);
    ctx->arena = (float*)p;
    ctx->arena_cap = need;
    ctx->ckdirty_halo.assign(need, 0);  // new memory: nothing known about any slot's tiles
    return PF_OK;
}

// Take n consecutive slots; returns the first slot index (or -1 with *rc set).
int take_slots(pf_ctx* ctx, int n, int* rc) {
    *rc = PF_OK;
    if (ctx->arena_used + n > ctx->arena_cap) {
        *rc = arena_reserve(ctx, std::max(ctx->arena_used + n, ctx->arena_cap + ctx->arena_cap / 2 + 8));
        if (*rc) return -1;
    }
    const int s0 = ctx->arena_used;
    ctx->arena_used += n;
    if ((int)ctx->ckact_halo.size() < ctx->arena_cap) ctx->ckact_halo.resize(ctx->arena_cap, 0);
    for (int i = s0; i < s0 + n; ++i) ctx->ckact_halo[i] = 0;  // no flags recorded for the new contents
    if ((int)ctx->ckdirty_halo.size() < ctx->arena_cap) ctx->ckdirty_halo.resize(ctx->arena_cap, 0);
    return s0;
}

// Keep the tile flags of the blocked forward's last launch (its act_out, describing the
// state it wrote into arena slot s) for the recompute that will start from that state.
int save_ckpt_flags(pf_ctx* ctx, int s) {
    const size_t nt = (size_t)std::max(diff_blocked_tiles(8, ctx->H, ctx->P), diff_blocked_tiles(4, ctx->H, ctx->P));
    if (ctx->ckact_cap < ctx->arena_cap) {
        void* p;
        int rc = dalloc(ctx, &p, nt * (size_t)ctx->arena_cap);
        if (rc) return rc;
        if (ctx->ckact) {
            CK(cudaMemcpyAsync(p, ctx->ckact, nt * (size_t)ctx->ckact_cap, cudaMemcpyDeviceToDevice, ctx->st));
            dfree(ctx, ctx->ckact);
        }
        ctx->ckact = (uint8_t*)p;
        ctx->ckact_cap = ctx->arena_cap;
    }
    CK(cudaMemcpyAsync(ctx->ckact + nt * s, ctx->fact[ctx->fl_par], nt, cudaMemcpyDeviceToDevice, ctx->st));
    ctx->ckact_halo[s] = ctx->fl_halo;
    return PF_OK;
}

bool is_ckpt_step(const pf_ctx* c, int t) {
    if ((t - c->tape_start) % c->K == 0) return true;
    for (auto& w : c->winds)
        if (w.from == t) return true;
    return false;
}

int choose_K(pf_ctx* ctx, int T) {
    if (ctx->tun.K > 0) return ctx->tun.K;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        free_b = 0;
    }
    const double sb = (double)diff_state_bytes(ctx);
    const int ne = (int)ctx->winds.size();
    // the per-epoch q cache (qcache_decide) is counted out of the tape's budget
    double cached = 0.0;
    for (float* b : ctx->qcache) cached += b ? 8.0 * (double)plane_elems(ctx) * sizeof(float) : 0.0;
    const double qbytes = 8.0 * (double)plane_elems(ctx) * sizeof(float) * ne;
    const double avail = (double)free_b + cached;
    const double budget = 0.6 * (avail + (double)ctx->arena_cap * sb) - (ctx->qcache_on ? qbytes - cached : 0.0);
    if ((double)(T + 1 + ne) * sb <= budget) return 1;  // keep every state: no recomputation
    int K = std::max(2, (int)std::ceil(std::sqrt((double)T)));
    return K;
}

// Device memory the tile tape and the q cache leave free for the caller: a sixteenth of
// the device, at least 16 GB.
size_t tape_keep_bytes(size_t total_b) { return std::max((size_t)16 << 30, total_b / 16); }

// Whether a taped forward keeps every epoch's q for the adjoint (saves the adjoint one
// prep per epoch): when they take at most 30% of the free memory, and, where a tile tape
// will be kept and the last one's need is known, when the tape's need (an eighth more)
// fits beside them with tape_keep_bytes left free. The tape
// saves a whole recompute, the cache one prep per epoch: the tape comes first. Buffers
// of a cache that is off are freed.
void qcache_decide(pf_ctx* ctx) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        free_b = 0;
    }
    const int ne = (int)ctx->winds.size();
    const double qb = 8.0 * (double)plane_elems(ctx) * sizeof(float);
    double cached = 0.0;
    for (float* b : ctx->qcache) cached += b ? qb : 0.0;
    // a tile tape's memory counts as free: ttape_begin sizes the tape after this
    const double held = ctx->ttape ? (double)ctx->ttape_cap * (double)ctx->ttape_blk : 0.0;
    bool on = qb * ne <= 0.3 * ((double)free_b + cached + held);
    const bool tape = ctx->form == PF_DIFF && ctx->tun.tape != 1 && ctx->tun.prep != 2 && choose_kernel(ctx) == 2;
    if (on && tape && ctx->ttape_need > 0) {
        const double need = (double)ctx->ttape_need * 1.125 * (double)ctx->ttape_need_blk;
        const double keep = (double)tape_keep_bytes(total_b);
        on = qb * ne - cached + need + keep + 2.0 * (1 << 30) <= (double)free_b + held;
    }
    ctx->qcache_on = on;
    if ((int)ctx->qcache.size() < ne) {
        ctx->qcache.resize(ne, nullptr);
        ctx->qcache_ver.resize(ne, -1);
        ctx->qcache_until.resize(ne, 0);
    }
    if (!ctx->qcache_on)
        for (float*& b : ctx->qcache)
            if (b) {
                if (ctx->q == b) use_q_buffer(ctx, ctx->q_own);
                dfree(ctx, b);
                b = nullptr;
            }
}

// steps from t until the next checkpoint step (exclusive bound t + result)
int steps_to_ckpt(const pf_ctx* c, int t) {
    if (!c->tape_valid) return 0x7fffffff;
    int n = 1;
    while (!is_ckpt_step(c, t + n)) ++n;
    return n;
}

int diff_steps(pf_ctx* ctx, int T) {
    const int end = ctx->step + T;
    const int kern = choose_kernel(ctx);
    ctx->fl_state = nullptr;  // the current state may have been set by other means
    ctx->fl_seed = nullptr;
    // with K == 1 every state is saved: blocked launches write all of them into
    // consecutive tape slots
    const bool all_states = ctx->tape_valid && ctx->K == 1;
    const bool rcq = ctx->tun.prep == 2;  // q recomputed inside the step kernels
    int pa_epoch = -1;
    PrepArgs pa{};
    while (ctx->step < end) {
        const int t = ctx->step;
        int rc;
        if (rcq) {
            const int e = epoch_of(ctx, t);
            if (e != pa_epoch) pa = prep_args(ctx, e, false);
            pa_epoch = e;
        } else if ((rc = ensure_q(ctx, epoch_of(ctx, t), std::min(end, next_epoch_start(ctx, t))))) {
            return rc;
        }
        int n = 1;
        // with the tile tape, launches of the adjoint's chunk from every checkpoint, as the
        // backward's recompute launches them (so that a record covers a recompute launch)
        const bool record = ctx->ttape_on && ctx->tape_valid && !all_states &&
                            (int)ctx->ttape_rec.size() < ctx->ttape_rec_cap;
        if (kern == 2) {
            n = std::min({record ? std::min(blocked_k(ctx), adjoint_blocked_max_steps()) : blocked_k(ctx), end - t,
                          next_epoch_start(ctx, t) - t});
            if (!all_states) n = std::min(n, steps_to_ckpt(ctx, t));
        }
        float* out = nullptr;
        float* all_out = nullptr;
        int ckpt_slot = -1;
        if (all_states) {
            const int s = take_slots(ctx, n, &rc);
            if (rc) return rc;
            for (int i = 0; i < n; ++i) {
                ctx->ckpts.push_back({t + 1 + i, s + i});
                ctx->ckdirty_halo[s + i] = 0;  // written whole: no dirty bits kept
            }
            all_out = slot_ptr(ctx, s);
        } else if (ctx->tape_valid && is_ckpt_step(ctx, t + n)) {
            const int s = take_slots(ctx, 1, &rc);
            if (rc) return rc;
            ctx->ckpts.push_back({t + n, s});
            out = slot_ptr(ctx, s);
            ckpt_slot = s;
        } else if (ctx->cur_ab == ctx->work[0] || ctx->cur_ab == ctx->work[1]) {
            out = (ctx->cur_ab == ctx->work[0]) ? ctx->work[1] : ctx->work[0];
        } else {
            // the state is in a checkpoint slot: the work buffer that was an input most
            // recently holds the most quiescent tiles' states already
            out = ctx->fl_in_at[1] > ctx->fl_in_at[0] ? ctx->work[1] : ctx->work[0];
        }
        if (kern == 2) {
            if ((rc = diff_blocked_launch(ctx, ctx->cur_ab, ctx->pc, n, out, all_out, false,
                                          all_states ? t + n : -1, false, rcq ? &pa : nullptr, ckpt_slot, -1,
                                          record)))
                return rc;
            if (ckpt_slot >= 0 && (rc = save_ckpt_flags(ctx, ckpt_slot))) return rc;
        } else {
            float* dst = out ? out : all_out;
            if (ckpt_slot >= 0) ctx->ckdirty_halo[ckpt_slot] = 0;  // written whole
            {
                LaunchScope ls(ctx, K_FSTEP);
                if (rcq)
                    launch_diff_step_rc(pa, ctx->pc, ctx->cur_ab, dst, ctx->st);
                else
                    launch_diff_step(ctx->H, ctx->W, ctx->P, ctx->pc, ctx->cur_ab, dst, ctx->q, ctx->st);
            }
            if ((rc = check_launch(ctx, "diff step"))) return rc;
        }
        ctx->cur_ab = out ? out : all_out + (size_t)(n - 1) * 2 * plane_elems(ctx);
        ctx->step = t + n;
    }
    return PF_OK;
}

void tape_reset(pf_ctx* ctx) {
    ctx->tape_valid = false;
    ctx->ttape_on = false;
    ctx->ttape_rec.clear();
    ctx->actrec_on = false;
    ctx->actrec_end.clear();
    ctx->ckpts.clear();
    // the current state may live in the arena: move it to a work buffer first
    if (ctx->arena && ctx->cur_ab && ctx->cur_ab >= ctx->arena &&
        ctx->cur_ab < ctx->arena + (size_t)ctx->arena_cap * 2 * plane_elems(ctx)) {
        float* w = ctx->work[0];
        cudaMemcpyAsync(w, ctx->cur_ab, diff_state_bytes(ctx), cudaMemcpyDeviceToDevice, ctx->st);
        ctx->cur_ab = w;
    }
    ctx->arena_used = 0;
}

// The tile tape of a checkpointed blocked run (pf_tuning.tape 0): blocks for the live
// tiles' states in the memory the backward does not need (its segment buffer, lambda,
// sigma and dL/dq, and the per-epoch q cache's buffers still to come are counted out)
// less tape_keep_bytes left to the caller, records for up to T
// launches. Without room, or for a run that keeps every state or runs the plain kernels,
// there is no tape and the backward recomputes its segments; launches the tape has no
// room for are recomputed too.
int ttape_begin(pf_ctx* ctx, int T) {
    ctx->ttape_on = false;
    ctx->ttape_rec.clear();
    if (ctx->tun.tape == 1 || ctx->K <= 1 || choose_kernel(ctx) != 2 || ctx->tun.prep == 2) return PF_OK;
    const int halo = blocked_k(ctx) <= 4 ? 4 : 8;
    const size_t ki = (size_t)(diff_blocked_box_rows() - 2 * halo);
    const size_t blk = 2 * ki * ki * sizeof(float);
    const size_t nt = (size_t)diff_blocked_tiles(halo, ctx->H, ctx->P);
    if (ctx->ttape_rec_cap < T) {
        for (void* p : {(void*)ctx->ttape_meta, (void*)ctx->ttape_lists})
            if (p) dfree(ctx, p);
        ctx->ttape_meta = nullptr;
        ctx->ttape_lists = nullptr;
        ctx->ttape_rec_cap = 0;
        void *pm, *pl;
        if (dalloc(ctx, &pm, 4 * sizeof(unsigned long long) * (size_t)T) != PF_OK) { cudaGetLastError(); return PF_OK; }
        ctx->ttape_meta = (unsigned long long*)pm;
        if (dalloc(ctx, &pl, sizeof(int) * nt * (size_t)T) != PF_OK) { cudaGetLastError(); return PF_OK; }
        ctx->ttape_lists = (int*)pl;
        ctx->ttape_rec_cap = T;
    }
    if (!ctx->ttape_used) {
        void *pu, *pi;
        if (dalloc(ctx, &pu, sizeof(unsigned long long)) != PF_OK) { cudaGetLastError(); return PF_OK; }
        ctx->ttape_used = (unsigned long long*)pu;
        if (dalloc(ctx, &pi, sizeof(int) * (size_t)std::max(diff_blocked_tiles(4, ctx->H, ctx->P),
                                                              diff_blocked_tiles(8, ctx->H, ctx->P))) != PF_OK)
            { cudaGetLastError(); return PF_OK; }
        ctx->ttape_inv = (int*)pi;
    }
    {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            cudaGetLastError();
            return PF_OK;
        }
        const size_t sb = diff_state_bytes(ctx), pe = plane_elems(ctx);
        // what the backward allocates later: the segment buffer, lambda and sigma
        // ping-pong, dL/dq, and a margin; and tape_keep_bytes
        // left to the caller. The tape's own memory counts as available.
        size_t later = (ctx->seg_cap < ctx->K ? (size_t)ctx->K * sb : 0) + 2 * sb + 2 * pe + 8 * pe * sizeof(float) +
                       ((size_t)2 << 30);
        if (ctx->lam[0]) later -= std::min(later, 2 * sb + 2 * pe + 8 * pe * sizeof(float));
        if (ctx->qcache_on)
            for (size_t e = 0; e < ctx->winds.size(); ++e)
                if (e >= ctx->qcache.size() || !ctx->qcache[e]) later += 8 * pe * sizeof(float);
        const size_t keep = tape_keep_bytes(total_b);
        const size_t avail = free_b + (ctx->ttape ? (size_t)ctx->ttape_cap * ctx->ttape_blk : 0);
        const size_t cap = avail > later + keep ? (avail - later - keep) / blk : 0;
        // the blocks to hold: what the last taped forward of this geometry needed and an
        // eighth more, or, before any is known, the room there is up to what T steps of
        // every tile would take
        const bool known = ctx->ttape_need > 0 && ctx->ttape_need_blk == blk;
        const size_t need = known ? (size_t)ctx->ttape_need : 0;
        size_t want = known ? std::min(cap, need + need / 8 + nt) : std::min(cap, (size_t)T * nt);
        // test hook: PF_TAPE_MAX_BLOCKS=n caps the tape at n blocks (read at every tape),
        // so that a run can be made to outgrow it and recompute its later launches
        bool capped = false;
        if (const char* e = getenv("PF_TAPE_MAX_BLOCKS")) {
            const long long m = atoll(e);
            if (m > 0 && (size_t)m < want) {
                want = (size_t)m;
                capped = true;
            }
        }
        // the tape is allocated again when it has another block size, when the run needs
        // its memory elsewhere now, when it is short of a known need that now fits, or
        // when it holds well over what is wanted (the rest is left to the caller)
        if (ctx->ttape && (ctx->ttape_blk != blk || cap < ctx->ttape_cap ||
                           (known && ctx->ttape_cap < need && want > ctx->ttape_cap) ||
                           ctx->ttape_cap > want + want / 4 || (capped && ctx->ttape_cap > want))) {
            dfree(ctx, ctx->ttape);
            ctx->ttape = nullptr;
            ctx->ttape_cap = 0;
        }
        if (!ctx->ttape) {
            if (want < nt) return PF_OK;
            void* p;
            if (dalloc(ctx, &p, want * blk) != PF_OK) {
                cudaGetLastError();
                return PF_OK;
            }
            ctx->ttape = (float*)p;
            ctx->ttape_cap = want;
            ctx->ttape_blk = blk;
        }
    }
    CK(cudaMemsetAsync(ctx->ttape_used, 0, sizeof(unsigned long long), ctx->st));
    ctx->ttape_on = true;
    return PF_OK;
}

// Start a fresh tape at the current step with the current state as checkpoint 0.
// The per-epoch q kept for the adjoint belongs to one tape: a new forward recomputes it.
int tape_begin(pf_ctx* ctx, int T) {
    tape_reset(ctx);
    for (long& v : ctx->qcache_ver) v = -1;
    for (int& v : ctx->qmask_state) v = 0;
    qcache_decide(ctx);
    ctx->q_key_epoch = -1;
    ctx->actrec_end.clear();
    ctx->actrec_on = true;
    ctx->K = choose_K(ctx, T);
    ctx->tape_start = ctx->step;
    ctx->t_p_h = ctx->p_h; ctx->t_c1 = ctx->c1; ctx->t_c2 = ctx->c2; ctx->t_a = ctx->a;
    ctx->t_pc = ctx->pc; ctx->t_l = ctx->l;
    ctx->t_version = ctx->version;
    const int want = ctx->K == 1 ? T + 1 : T / ctx->K + (int)ctx->winds.size() + 2;
    int rc = arena_reserve(ctx, want);
    if (rc) return rc;
    const int s = take_slots(ctx, 1, &rc);
    if (rc) return rc;
    float* s0 = slot_ptr(ctx, s);
    CK(cudaMemcpyAsync(s0, ctx->cur_ab, diff_state_bytes(ctx), cudaMemcpyDeviceToDevice, ctx->st));
    ctx->ckdirty_halo[s] = 0;  // written whole
    ctx->cur_ab = s0;
    ctx->ckpts.push_back({ctx->step, s});
    ctx->tape_valid = true;
    if ((rc = ttape_begin(ctx, T))) return rc;
    return PF_OK;
}

int write_diff_out(pf_ctx* ctx, void* out) {
    if (!out) return PF_OK;
    {
        LaunchScope ls(ctx, K_MISC);
        launch_diff_unpack(ctx->cur_ab, ctx->H, ctx->W, ctx->P, (float*)out, ctx->st);
    }
    return check_launch(ctx, "diff unpack");
}

int write_discrete_out(pf_ctx* ctx, void* out) {
    if (!out) return PF_OK;
    CK(cudaMemcpy2DAsync(out, ctx->W, ctx->S[ctx->scur], ctx->P, ctx->W, (size_t)ctx->R * ctx->H,
                         cudaMemcpyDeviceToDevice, ctx->st));
    return PF_OK;
}

int validate_states(pf_ctx* ctx, const uint8_t* S, size_t n) {
    CK(cudaMemsetAsync(ctx->dflags + 1, 0, sizeof(int), ctx->st));
    {
        LaunchScope ls(ctx, K_MISC);
        launch_validate_states(S, n, ctx->dflags + 1, ctx->st);
    }
    int rc = check_launch(ctx, "validate states");
    if (rc) return rc;
    CK(cudaMemcpyAsync(ctx->hflags + 1, ctx->dflags + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (ctx->hflags[1]) return fail(ctx, PF_EINVAL, "state array holds codes other than 0..3");
    return PF_OK;
}

}  // namespace

// Start recording a discrete trajectory for the accumulator path: zero the accumulator,
// keep the initial state (now in S[0]) and the parameters it runs with.
int dca_record(pf_ctx* ctx) {
    const size_t sb = (size_t)ctx->R * ctx->H * ctx->P;
    int rc;
    for (uint8_t** b : {&ctx->dca_S0, &ctx->dca_S[0], &ctx->dca_S[1]}) {
        if (*b) continue;
        void* p;
        if ((rc = dalloc(ctx, &p, sb))) return rc;
        *b = (uint8_t*)p;
    }
    CK(cudaMemcpyAsync(ctx->dca_S0, ctx->S[0], sb, cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaMemsetAsync(ctx->acc, 0, sb / ctx->P * ctx->W * sizeof(float), ctx->st));
    ctx->t_p_h = ctx->p_h; ctx->t_c1 = ctx->c1; ctx->t_c2 = ctx->c2; ctx->t_a = ctx->a;
    ctx->t_pc = ctx->pc; ctx->t_l = ctx->l;
    ctx->dca_version = ctx->version;
    ctx->dca_valid = true;
    return PF_OK;
}

// =================================================================== C ABI
extern "C" {

const char* pf_version(void) { return "libpfire 0.1 (sm_103a)"; }

const char* pf_last_error(const pf_ctx* ctx) { return ctx ? ctx->err.c_str() : g_last_error.c_str(); }

int pf_create(pf_ctx** out, int H, int W, int form, int realisations, uint64_t seed, void* cuda_stream) {
    if (!out) return fail(nullptr, PF_EINVAL, "pf_create: out is NULL");
    *out = nullptr;
    if (H < 1 || W < 1 || H > 65536 || W > 65536)
        return fail(nullptr, PF_EINVAL, "pf_create: grid %dx%d outside 1..65536", H, W);
    if (form != PF_DISCRETE && form != PF_DIFF) return fail(nullptr, PF_EINVAL, "pf_create: unknown form %d", form);
    if (realisations < 1) return fail(nullptr, PF_EINVAL, "pf_create: realisations must be >= 1");
    if (form == PF_DIFF && realisations != 1)
        return fail(nullptr, PF_EINVAL, "pf_create: the differentiable form takes realisations = 1");
    if ((uint64_t)H * (uint64_t)W * (uint64_t)realisations >= (1ull << 32))
        return fail(nullptr, PF_EINVAL, "pf_create: H*W*R must be below 2^32");
    pf_ctx* ctx = new pf_ctx();
    ctx->pool = g_ctx_pool;
    ctx->H = H; ctx->W = W; ctx->P = pitch_of(W); ctx->form = form; ctx->R = realisations;
    ctx->seed = seed;
    ctx->st = (cudaStream_t)cuda_stream;
    ctx->winds.push_back({0, nullptr, nullptr});
    {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
            ctx->nsm = nsm;
        cudaGetLastError();
    }
    int rc = PF_OK;
    const size_t pe = plane_elems(ctx);
#define ALLOC(ptr, bytes)                                         \
    do {                                                          \
        void* p_ = nullptr;                                       \
        rc = dalloc(ctx, &p_, (bytes));                           \
        if (rc) goto failed;                                      \
        ptr = (decltype(ptr))p_;                                  \
    } while (0)
    ALLOC(ctx->q, 8 * pe * sizeof(float));
    ctx->q_own = ctx->q;
    if (cudaMemsetAsync(ctx->q, 0, 8 * pe * sizeof(float), ctx->st) != cudaSuccess) goto cuda_failed;
    ALLOC(ctx->dflags, 16 * sizeof(int));
    ALLOC(ctx->dskip, K_NKINDS * sizeof(unsigned long long));
    ALLOC(ctx->dties, 8 * sizeof(unsigned long long));
    if (cudaMemsetAsync(ctx->dties, 0, 8 * sizeof(unsigned long long), ctx->st) != cudaSuccess) goto cuda_failed;
    if (cudaMallocHost((void**)&ctx->hflags, 16 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        rc = fail(ctx, PF_ENOMEM, "pinned flag allocation failed");
        goto failed;
    }
    if (cudaMemsetAsync(ctx->dflags, 0, 16 * sizeof(int), ctx->st) != cudaSuccess) goto cuda_failed;
    if (cudaMemsetAsync(ctx->dskip, 0, K_NKINDS * sizeof(unsigned long long), ctx->st) != cudaSuccess)
        goto cuda_failed;
    if (form == PF_DISCRETE) {
        const size_t sb = (size_t)realisations * pe;
        ALLOC(ctx->S[0], sb);
        ALLOC(ctx->S[1], sb);
        if (cudaMemsetAsync(ctx->S[0], 0, sb, ctx->st) != cudaSuccess) goto cuda_failed;
        if (cudaMemsetAsync(ctx->S[1], 0, sb, ctx->st) != cudaSuccess) goto cuda_failed;
        ctx->tmap_ok = encode_state_map(ctx, &ctx->tmapS[0], ctx->S[0]) &&
                       encode_state_map(ctx, &ctx->tmapS[1], ctx->S[1]);
    } else {
        ctx->tmapQ_ok = diff_blocked_configure() == 0 &&
                        encode_f32_3d(&ctx->tmapQ, ctx->q, ctx->P, H, 8, diff_blocked_box_cols(),
                                      diff_blocked_box_rows(), 8);
        cudaGetLastError();
        ALLOC(ctx->work[0], diff_state_bytes(ctx));
        ALLOC(ctx->work[1], diff_state_bytes(ctx));
        ALLOC(ctx->burn, (size_t)H * W);
        ALLOC(ctx->tile_list, (size_t)adjoint_blocked_tiles(H, ctx->P) * sizeof(int));
        ALLOC(ctx->adeadcnt, (size_t)adjoint_blocked_tiles(H, ctx->P));
        ALLOC(ctx->gqdirty, (size_t)adjoint_blocked_tiles(H, ctx->P));
        {
            const size_t nt = (size_t)std::max(diff_blocked_tiles(8, H, ctx->P), diff_blocked_tiles(4, H, ctx->P));
            ALLOC(ctx->fact[0], nt);
            ALLOC(ctx->fact[1], nt);
            ALLOC(ctx->fqrun, nt);
            ALLOC(ctx->flist, nt * sizeof(int));
        }
        if (cudaMemsetAsync(ctx->work[0], 0, diff_state_bytes(ctx), ctx->st) != cudaSuccess) goto cuda_failed;
        if (cudaMemsetAsync(ctx->work[1], 0, diff_state_bytes(ctx), ctx->st) != cudaSuccess) goto cuda_failed;
        if (cudaMemsetAsync(ctx->burn, 1, (size_t)H * W, ctx->st) != cudaSuccess) goto cuda_failed;
        ctx->cur_ab = ctx->work[0];
    }
    if (cudaStreamSynchronize(ctx->st) != cudaSuccess) goto cuda_failed;
    *out = ctx;
    return PF_OK;
cuda_failed:
    rc = fail(ctx, PF_ECUDA, "pf_create: %s", cudaGetErrorString(cudaGetLastError()));
failed : {
    std::string msg = ctx->err;
    pf_destroy(ctx);
    g_last_error = msg;
    return rc;
}
#undef ALLOC
}

void pf_destroy(pf_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->st);
    if (ctx->cst) {
        cudaStreamSynchronize(ctx->cst);
        cudaStreamDestroy(ctx->cst);
    }
    for (auto& w : ctx->winds)
        if (w.ready) cudaEventDestroy(w.ready);
    for (auto& r : ctx->prof) {
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    for (void* p : ctx->allocs) {
        if (ctx->pool) cudaFreeAsync(p, ctx->st);
        else cudaFree(p);
    }
    if (ctx->hflags) cudaFreeHost(ctx->hflags);
    cudaGetLastError();
    delete ctx;
}

int pf_set_params(pf_ctx* ctx, float p_h, float c1, float c2, float a, float p_continue, float l_m) {
    if (!ctx) return fail(nullptr, PF_EINVAL, "pf_set_params: ctx is NULL");
    const float v[6] = {p_h, c1, c2, a, p_continue, l_m};
    for (float x : v)
        if (!std::isfinite(x)) return fail(ctx, PF_EINVAL, "pf_set_params: non-finite parameter");
    if (p_h < 0.f) return fail(ctx, PF_EINVAL, "pf_set_params: p_h must be >= 0");
    if (p_continue < 0.f || p_continue > 1.f) return fail(ctx, PF_EINVAL, "pf_set_params: p_continue outside [0,1]");
    if (!(l_m > 0.f)) return fail(ctx, PF_EINVAL, "pf_set_params: l must be > 0");
    ctx->p_h = p_h; ctx->c1 = c1; ctx->c2 = c2; ctx->a = a; ctx->pc = p_continue; ctx->l = l_m;
    ctx->version++;
    tape_reset(ctx);
    return PF_OK;
}

static int copy_field(pf_ctx* ctx, float** dst, const float* src) {
    const size_t bytes = (size_t)ctx->H * ctx->W * sizeof(float);
    if (!src) {
        if (*dst) dfree(ctx, *dst);
        *dst = nullptr;
        return PF_OK;
    }
    if (!*dst) {
        void* p;
        int rc = dalloc(ctx, &p, bytes);
        if (rc) return rc;
        *dst = (float*)p;
    }
    CK(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyDeviceToDevice, ctx->st));
    return PF_OK;
}

// An H*W buffer for a wind epoch: one of a dropped epoch's (the stream orders its reuse
// after the work that read it), else a new allocation.
static int wind_buffer(pf_ctx* ctx, float** out) {
    if (!ctx->wind_pool.empty()) {
        *out = ctx->wind_pool.back();
        ctx->wind_pool.pop_back();
        return PF_OK;
    }
    void* p;
    int rc = dalloc(ctx, &p, (size_t)ctx->H * ctx->W * sizeof(float));
    if (rc) return rc;
    *out = (float*)p;
    return PF_OK;
}

// Drop the wind epochs after the first. Their buffers go to the pool; an upload still in
// flight is ordered before any later work of the context's stream (which reuses them).
static int drop_epochs(pf_ctx* ctx) {
    for (size_t i = 1; i < ctx->winds.size(); ++i) {
        Epoch& w = ctx->winds[i];
        if (w.ready) {
            CK(cudaStreamWaitEvent(ctx->st, w.ready, 0));
            cudaEventDestroy(w.ready);
        }
        if (w.V) ctx->wind_pool.push_back(w.V);
        if (w.th) ctx->wind_pool.push_back(w.th);
    }
    ctx->winds.resize(1);
    return PF_OK;
}

static int validate_fields(pf_ctx* ctx, const float* const* f, const float* lo, int n) {
    const size_t cells = (size_t)ctx->H * ctx->W;
    CK(cudaMemsetAsync(ctx->dflags + 1, 0, sizeof(int), ctx->st));
    for (int i = 0; i < n; ++i) {
        if (!f[i]) continue;
        LaunchScope ls(ctx, K_MISC);
        launch_validate_fields(f[i], cells, lo[i], i, ctx->dflags + 1, ctx->st);
    }
    int rc = check_launch(ctx, "validate fields");
    if (rc) return rc;
    CK(cudaMemcpyAsync(ctx->hflags + 1, ctx->dflags + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return ctx->hflags[1];
}

int pf_set_env(pf_ctx* ctx, const float* E, const float* p_veg, const float* p_den, const float* V_w,
               const float* theta_w_deg) {
    if (!ctx) return fail(nullptr, PF_EINVAL, "pf_set_env: ctx is NULL");
    const float* f[5] = {E, p_veg, p_den, V_w, theta_w_deg};
    const float lo[5] = {-INFINITY, -1.0f, -1.0f, -INFINITY, -INFINITY};
    const char* names[5] = {"E", "p_veg", "p_den", "V_w", "theta_w"};
    int bad = validate_fields(ctx, f, lo, 5);
    if (bad < 0) return bad;
    if (bad) {
        std::string which;
        for (int i = 0; i < 5; ++i)
            if (bad & (1 << i)) which += std::string(which.empty() ? "" : ", ") + names[i];
        return fail(ctx, PF_EINVAL, "pf_set_env: invalid values (NaN/inf, or p_veg/p_den < -1) in %s", which.c_str());
    }
    int rc;
    if ((rc = copy_field(ctx, &ctx->E, E))) return rc;
    if ((rc = copy_field(ctx, &ctx->pveg, p_veg))) return rc;
    if ((rc = copy_field(ctx, &ctx->pden, p_den))) return rc;
    if ((rc = drop_epochs(ctx))) return rc;
    if ((rc = copy_field(ctx, &ctx->winds[0].V, V_w))) return rc;
    if ((rc = copy_field(ctx, &ctx->winds[0].th, theta_w_deg))) return rc;
    ctx->version++;
    tape_reset(ctx);
    return PF_OK;
}

int pf_set_slope(pf_ctx* ctx, const float* slope_deg) {
    if (!ctx) return fail(nullptr, PF_EINVAL, "pf_set_slope: ctx is NULL");
    if (!slope_deg) {
        if (ctx->slope) dfree(ctx, ctx->slope);
        ctx->slope = nullptr;
    } else {
        const size_t n = (size_t)ctx->H * ctx->W * 9;
        CK(cudaMemsetAsync(ctx->dflags + 1, 0, sizeof(int), ctx->st));
        {
            LaunchScope ls(ctx, K_MISC);
            launch_validate_fields(slope_deg, n, -INFINITY, 0, ctx->dflags + 1, ctx->st);
        }
        int rc = check_launch(ctx, "validate slope");
        if (rc) return rc;
        CK(cudaMemcpyAsync(ctx->hflags + 1, ctx->dflags + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        if (ctx->hflags[1]) return fail(ctx, PF_EINVAL, "pf_set_slope: NaN or infinite slope values");
        if (!ctx->slope) {
            void* p;
            if ((rc = dalloc(ctx, &p, n * sizeof(float)))) return rc;
            ctx->slope = (float*)p;
        }
        CK(cudaMemcpyAsync(ctx->slope, slope_deg, n * sizeof(float), cudaMemcpyDeviceToDevice, ctx->st));
    }
    ctx->version++;
    tape_reset(ctx);
    return PF_OK;
}

int pf_set_wind(pf_ctx* ctx, const float* V_w, const float* theta_w_deg, int from_step) {
    if (!ctx) return fail(nullptr, PF_EINVAL, "pf_set_wind: ctx is NULL");
    if (from_step <= ctx->winds.back().from)
        return fail(ctx, PF_EINVAL, "pf_set_wind: from_step %d must exceed the last epoch's start %d", from_step,
                    ctx->winds.back().from);
    const float* f[2] = {V_w, theta_w_deg};
    const float lo[2] = {-INFINITY, -INFINITY};
    int bad = validate_fields(ctx, f, lo, 2);
    if (bad < 0) return bad;
    if (bad) return fail(ctx, PF_EINVAL, "pf_set_wind: NaN or infinite wind values");
    Epoch e{from_step, nullptr, nullptr};
    int rc;
    if (V_w && (rc = wind_buffer(ctx, &e.V))) return rc;
    if (theta_w_deg && (rc = wind_buffer(ctx, &e.th))) return rc;
    if ((rc = copy_field(ctx, &e.V, V_w))) return rc;
    if ((rc = copy_field(ctx, &e.th, theta_w_deg))) return rc;
    ctx->winds.push_back(e);
    if (ctx->tape_valid && from_step <= ctx->step) tape_reset(ctx);
    return PF_OK;
}

int pf_set_wind_async(pf_ctx* ctx, const float* V_w, const float* theta_w_deg, int from_step) {
    if (!ctx) return fail(nullptr, PF_EINVAL, "pf_set_wind_async: ctx is NULL");
    if (from_step <= ctx->winds.back().from)
        return fail(ctx, PF_EINVAL, "pf_set_wind_async: from_step %d must exceed the last epoch's start %d",
                    from_step, ctx->winds.back().from);
    if (!ctx->cst) CK(cudaStreamCreateWithFlags(&ctx->cst, cudaStreamNonBlocking));
    Epoch e{from_step, nullptr, nullptr};
    int rc;
    if (V_w && (rc = wind_buffer(ctx, &e.V))) return rc;
    if (theta_w_deg && (rc = wind_buffer(ctx, &e.th))) return rc;
    CK(cudaEventCreateWithFlags(&e.ready, cudaEventDisableTiming));
    ctx->winds.push_back(e);  // from here on the event is owned (and destroyed) with the epoch
    // the buffers may come from the pool: the copy waits for the work already queued on
    // the context's stream, which may still read them
    CK(cudaEventRecord(e.ready, ctx->st));
    CK(cudaStreamWaitEvent(ctx->cst, e.ready, 0));
    const size_t cells = (size_t)ctx->H * ctx->W;
    if (V_w) CK(cudaMemcpyAsync(e.V, V_w, cells * sizeof(float), cudaMemcpyDefault, ctx->cst));
    if (theta_w_deg) CK(cudaMemcpyAsync(e.th, theta_w_deg, cells * sizeof(float), cudaMemcpyDefault, ctx->cst));
    // checked on the copy stream and reported by the next synchronising call (device_error);
    // counted as misc launches, untimed (the profile's events are on the context's stream)
    if (e.V) launch_validate_fields(e.V, cells, -INFINITY, 0, ctx->dflags + 3, ctx->cst);
    if (e.th) launch_validate_fields(e.th, cells, -INFINITY, 1, ctx->dflags + 3, ctx->cst);
    ctx->launches[K_MISC] += (e.V ? 1 : 0) + (e.th ? 1 : 0);
    if ((rc = check_launch(ctx, "validate uploaded wind"))) return rc;
    CK(cudaEventRecord(e.ready, ctx->cst));
    if (ctx->tape_valid && from_step <= ctx->step) tape_reset(ctx);
    return PF_OK;
}

int pf_wait(pf_ctx* ctx) {
    if (!ctx) return fail(nullptr, PF_EINVAL, "pf_wait: ctx is NULL");
    return device_error(ctx);
}

namespace {

// Tile geometry of the blocked discrete kernel: TH interior rows, KH halo rows (>= the
// steps of one launch). Re-encodes both state tensor maps for the new box.
int set_discrete_tiles(pf_ctx* ctx, int TH, int KH) {
    if (ctx->form != PF_DISCRETE || (ctx->TH == TH && ctx->KH == KH)) return PF_OK;
    const int oTH = ctx->TH, oKH = ctx->KH;
    ctx->TH = TH;
    ctx->KH = KH;
    if (!encode_state_map(ctx, &ctx->tmapS[0], ctx->S[0]) || !encode_state_map(ctx, &ctx->tmapS[1], ctx->S[1])) {
        ctx->TH = oTH;
        ctx->KH = oKH;
        ctx->tmap_ok = encode_state_map(ctx, &ctx->tmapS[0], ctx->S[0]) &&
                       encode_state_map(ctx, &ctx->tmapS[1], ctx->S[1]);
        return fail(ctx, PF_ECUDA, "tensor map encoding for %d-row tiles failed", TH);
    }
    return PF_OK;
}

int apply_tuning(pf_ctx* ctx, const pf_tuning* t) {
    if (t->kernel < 0 || t->kernel > 2) return fail(ctx, PF_EINVAL, "pf_set_tuning: kernel must be 0, 1 or 2");
    if (t->k < 0 || t->k > 16) return fail(ctx, PF_EINVAL, "pf_set_tuning: k must be in 0..16");
    if (t->K < 0) return fail(ctx, PF_EINVAL, "pf_set_tuning: K must be >= 0");
    if (t->prep < 0 || t->prep > 2) return fail(ctx, PF_EINVAL, "pf_set_tuning: prep must be 0, 1 or 2");
    if (t->tape < 0 || t->tape > 1) return fail(ctx, PF_EINVAL, "pf_set_tuning: tape must be 0 or 1");
    if (t->tile_rows != 0 && t->tile_rows != 16 && t->tile_rows != 32 && t->tile_rows != 64 && t->tile_rows != 128)
        return fail(ctx, PF_EINVAL, "pf_set_tuning: tile_rows must be 0, 16, 32, 64 or 128");
    if (ctx->form == PF_DISCRETE) {
        const int rc = set_discrete_tiles(ctx, t->tile_rows ? t->tile_rows : 64,
                                          t->k ? std::min(t->k, discrete_blocked_max_k()) : 16);
        if (rc) return rc;
    }
    ctx->tun = *t;
    return PF_OK;
}

// ------------------------------------------------------------- tuning cache
// One line per tuned configuration: "<key>\t<kernel> <k> <prep> <tile_rows> <K>". The
// newest line of a key wins; a file that cannot be read or written is skipped.
std::string tune_cache_path() {
    const char* e = getenv("PF_TUNE_CACHE");
    if (e) return (e[0] == '\0' || strcmp(e, "off") == 0) ? std::string() : std::string(e);
    std::string dir;
    const char* x = getenv("XDG_CACHE_HOME");
    const char* h = getenv("HOME");
    if (x && x[0])
        dir = x;
    else if (h && h[0])
        dir = std::string(h) + "/.cache";
    else
        return std::string();
    return dir + "/pfire/tuning.tsv";
}

// (GPU model, compute capability, SM count, search, form, H, W, R, T)
std::string tune_key(const pf_ctx* ctx, const char* what, int T) {
    cudaDeviceProp prop;
    int dev = 0;
    std::string gpu = "unknown";
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
        char b[320];
        snprintf(b, sizeof b, "%s sm_%d%d x%d", prop.name, prop.major, prop.minor, prop.multiProcessorCount);
        gpu = b;
    } else {
        cudaGetLastError();
    }
    for (char& ch : gpu)
        if (ch == '\t' || ch == '\n' || ch == '|') ch = ' ';
    char b[160];
    snprintf(b, sizeof b, "|%s|%s|H=%d|W=%d|R=%d|T=%d", what, ctx->form == PF_DIFF ? "diff" : "discrete", ctx->H,
             ctx->W, ctx->R, T);
    return gpu + b;
}

bool tune_cache_get(const std::string& key, pf_tuning* t) {
    const std::string path = tune_cache_path();
    if (path.empty()) return false;
    std::ifstream f(path);
    if (!f) return false;
    std::string line;
    bool found = false;
    while (std::getline(f, line)) {
        const size_t tab = line.find('\t');
        if (tab != key.size() || line.compare(0, tab, key) != 0) continue;
        std::istringstream v(line.substr(tab + 1));
        pf_tuning x{};
        if (v >> x.kernel >> x.k >> x.prep >> x.tile_rows >> x.K) {
            *t = x;
            found = true;
        }
    }
    return found;
}

void tune_cache_put(const std::string& key, const pf_tuning& t) {
    const std::string path = tune_cache_path();
    if (path.empty()) return;
    for (size_t i = 1; i < path.size(); ++i)  // parent directories, mode 0755
        if (path[i] == '/') mkdir(path.substr(0, i).c_str(), 0755);
    std::ofstream f(path, std::ios::app);
    if (f) f << key << '\t' << t.kernel << ' ' << t.k << ' ' << t.prep << ' ' << t.tile_rows << ' ' << t.K << '\n';
}

// state of a probe run: S_init copied (discrete) or initialised (differentiable)
int probe_start(pf_ctx* ctx, const uint8_t* S_init) {
    ctx->step = 0;
    if (ctx->form == PF_DISCRETE) {
        ctx->scur = 0;
        if (cudaMemcpy2DAsync(ctx->S[0], ctx->P, S_init, ctx->W, ctx->W, (size_t)ctx->R * ctx->H,
                              cudaMemcpyDeviceToDevice, ctx->st) != cudaSuccess)
            return fail(ctx, PF_ECUDA, "pf_autotune: state copy failed");
    } else {
        launch_diff_init(S_init, ctx->H, ctx->W, ctx->P, ctx->work[0], ctx->burn, ctx->st);
        ctx->cur_ab = ctx->work[0];
        ctx->version++;  // every materialising candidate pays for its own prep
    }
    return PF_OK;
}

}  // namespace

int pf_set_tuning(pf_ctx* ctx, const pf_tuning* t) {
    if (!ctx || !t) return fail(ctx, PF_EINVAL, "pf_set_tuning: NULL argument");
    return apply_tuning(ctx, t);
}

int pf_memory_stats(pf_ctx* ctx, pf_memory_stats_t* out) {
    if (!ctx || !out) return fail(ctx, PF_EINVAL, "pf_memory_stats: NULL argument");
    *out = pf_memory_stats_t{};
    const size_t sb = ctx->form == PF_DIFF ? diff_state_bytes(ctx) : 0;
    out->checkpoint_bytes = (long long)ctx->arena_cap * (long long)sb;
    out->segment_bytes = (long long)ctx->seg_cap * (long long)sb;
    for (float* b : ctx->qcache)
        if (b) out->qcache_bytes += 8LL * (long long)plane_elems(ctx) * (long long)sizeof(float);
    out->tape_bytes = ctx->ttape ? (long long)(ctx->ttape_cap * ctx->ttape_blk) : 0;
    out->K = ctx->K;
    out->tape_short = ctx->ttape_short ? 1 : 0;
    out->allocations = ctx->n_allocs;
    out->frees = ctx->n_frees;
    const size_t nr = ctx->ttape_rec.size();
    out->tape_launches = (int)nr;
    if (ctx->ttape_used && nr > 0) {
        unsigned long long used = 0;
        std::vector<unsigned long long> meta(4 * nr);
        CK(cudaMemcpyAsync(&used, ctx->ttape_used, sizeof(used), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaMemcpyAsync(meta.data(), ctx->ttape_meta, meta.size() * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        out->tape_used_bytes = (long long)(std::min<unsigned long long>(used, ctx->ttape_cap) * ctx->ttape_blk);
        for (size_t L = 0; L < nr; ++L) out->tape_recorded += meta[4 * L + 3] ? 1 : 0;
    }
    return PF_OK;
}

int pf_get_tuning(const pf_ctx* ctx, pf_tuning* t) {
    if (!ctx || !t) return fail(nullptr, PF_EINVAL, "pf_get_tuning: NULL argument");
    *t = ctx->tun;
    t->kernel = choose_kernel(ctx);
    if (t->k == 0) t->k = blocked_k(ctx);
    if (t->K == 0) t->K = ctx->K;
    if (t->prep == 0) t->prep = 1;
    t->tile_rows = ctx->form == PF_DISCRETE ? ctx->TH : 0;
    return PF_OK;
}

int pf_autotune(pf_ctx* ctx, const uint8_t* S_init, int T_probe, pf_tuning* chosen) {
    if (!ctx) return fail(nullptr, PF_EINVAL, "pf_autotune: ctx is NULL");
    if (!S_init) return fail(ctx, PF_EINVAL, "pf_autotune: S_init is NULL");
    if (T_probe < 1) return fail(ctx, PF_EINVAL, "pf_autotune: T_probe must be >= 1");
    int rc = validate_states(ctx, S_init, (size_t)ctx->R * ctx->H * ctx->W);
    if (rc) return rc;
    const pf_tuning saved = ctx->tun;
    const std::string key = tune_key(ctx, "launch", T_probe);
    pf_tuning hit;
    if (tune_cache_get(key, &hit) && hit.kernel >= 1) {
        hit.K = saved.K;  // this search leaves K alone
        hit.profile = saved.profile;
        hit.tape = saved.tape;
        if (apply_tuning(ctx, &hit) == PF_OK) {
            if (chosen) pf_get_tuning(ctx, chosen);
            return PF_OK;
        }
        ctx->tun = saved;
    }
    // candidates: q materialised per wind epoch (prep 1) or recomputed inside the step
    // kernels (prep 2), each with the plain per-step kernels and the temporal-blocked ones
    // at several depths k (the differentiable blocked kernel switches to its 4-cell halo
    // for k <= 4; the discrete one also takes 32, 64 or 128 interior rows per tile)
    std::vector<pf_tuning> cand;
    for (int prep : {1, 2}) {
        cand.push_back({1, 1, saved.K, saved.profile, prep, 0, saved.tape});
        if (ctx->form == PF_DISCRETE) {
            if (ctx->tmap_ok)
                for (int k : {4, 8, 12})
                    for (int rows : {32, 64, 128}) cand.push_back({2, k, saved.K, saved.profile, prep, rows, saved.tape});
        } else if (ctx->tmapQ_ok) {
            for (int k : {2, 4, 6, 8}) cand.push_back({2, k, saved.K, saved.profile, prep, 0, saved.tape});
        }
    }
    tape_reset(ctx);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, PF_ECUDA, "pf_autotune: event creation failed");
    }
    float best_ms = 0.f;
    int best = -1;
    for (int rep = 0; rep < 2 && rc == PF_OK; ++rep)  // first pass warms every variant up
        for (size_t c = 0; c < cand.size() && rc == PF_OK; ++c) {
            if ((rc = apply_tuning(ctx, &cand[c])) || (rc = probe_start(ctx, S_init))) break;
            cudaEventRecord(e0, ctx->st);
            rc = ctx->form == PF_DISCRETE ? run_discrete(ctx, T_probe) : diff_steps(ctx, T_probe);
            cudaEventRecord(e1, ctx->st);
            if (rc) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = fail(ctx, PF_ECUDA, "pf_autotune: %s", cudaGetErrorString(cudaGetLastError()));
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep == 1 && (best < 0 || ms < best_ms)) {
                best_ms = ms;
                best = (int)c;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->step = 0;
    if (rc) {
        apply_tuning(ctx, &saved);
        return rc;
    }
    if ((rc = apply_tuning(ctx, &cand[best]))) return rc;
    tune_cache_put(key, cand[best]);
    if (chosen) pf_get_tuning(ctx, chosen);
    return PF_OK;
}

int pf_autotune_ckpt(pf_ctx* ctx, const uint8_t* S_init, int T, int* K_chosen) {
    if (!ctx) return fail(nullptr, PF_EINVAL, "pf_autotune_ckpt: ctx is NULL");
    if (!S_init) return fail(ctx, PF_EINVAL, "pf_autotune_ckpt: S_init is NULL");
    if (ctx->form != PF_DIFF) return fail(ctx, PF_ESTATE, "pf_autotune_ckpt: only the differentiable form is taped");
    if (T < 1) return fail(ctx, PF_EINVAL, "pf_autotune_ckpt: T must be >= 1");
    int rc = validate_states(ctx, S_init, (size_t)ctx->H * ctx->W);
    if (rc) return rc;
    const pf_tuning saved = ctx->tun;
    const std::string key = tune_key(ctx, "K", T);
    pf_tuning hit;
    if (tune_cache_get(key, &hit) && hit.K >= 0) {
        ctx->tun.K = hit.K;
        if (K_chosen) *K_chosen = hit.K;
        return PF_OK;
    }
    // the memory rule (0), and intervals that are multiples of the blocked kernel's depth
    // (no launch is cut short at a checkpoint) around the interval it picks
    ctx->tun.K = 0;
    tape_reset(ctx);
    qcache_decide(ctx);
    const int K0 = choose_K(ctx, T);
    std::vector<int> cand = {0};
    if (K0 > 1) {
        const int k = choose_kernel(ctx) == 2 ? blocked_k(ctx) : 1;
        for (int K : {k * ((K0 + k - 1) / k), k * (K0 / k), k * ((2 * K0 + k - 1) / k)})
            if (K >= 2 && K != K0 && std::find(cand.begin(), cand.end(), K) == cand.end()) cand.push_back(K);
    }
    std::vector<double> t_ms(cand.size(), 0.0);
    double grads[4];
    for (int rep = 0; rep < 2 && rc == PF_OK && cand.size() > 1; ++rep)  // first pass warms up
        for (size_t c = 0; c < cand.size() && rc == PF_OK; ++c) {
            ctx->tun.K = cand[c];
            if (cudaStreamSynchronize(ctx->st) != cudaSuccess) {
                rc = fail(ctx, PF_ECUDA, "pf_autotune_ckpt: %s", cudaGetErrorString(cudaGetLastError()));
                break;
            }
            const auto t0 = std::chrono::steady_clock::now();
            if ((rc = pf_forward(ctx, S_init, T, nullptr))) break;
            if ((rc = pf_backward(ctx, nullptr, nullptr, grads, nullptr, nullptr))) break;
            const auto t1 = std::chrono::steady_clock::now();
            if (rep == 1) t_ms[c] = std::chrono::duration<double, std::milli>(t1 - t0).count();
        }
    ctx->tun = saved;
    tape_reset(ctx);
    if (rc) return rc;
    size_t best = 0;
    for (size_t c = 1; c < cand.size(); ++c)
        if (t_ms[c] < t_ms[best]) best = c;
    ctx->tun.K = cand[best];
    // a segment buffer sized for a larger candidate is given back: the next backward
    // allocates the chosen interval's
    if (ctx->seg_buf && ctx->seg_cap > std::max(cand[best], 2)) {
        dfree(ctx, ctx->seg_buf);
        ctx->seg_buf = nullptr;
        ctx->seg_cap = 0;
        ctx->seg_halo = 0;
    }
    tune_cache_put(key, ctx->tun);
    if (K_chosen) *K_chosen = cand[best];
    return PF_OK;
}

int pf_forward(pf_ctx* ctx, const uint8_t* S_init, int T, void* S_out) {
    if (!ctx) return fail(nullptr, PF_EINVAL, "pf_forward: ctx is NULL");
    if (!S_init) return fail(ctx, PF_EINVAL, "pf_forward: S_init is NULL");
    if (T < 0) return fail(ctx, PF_EINVAL, "pf_forward: T must be >= 0");
    const size_t n = (size_t)ctx->R * ctx->H * ctx->W;
    int rc = validate_states(ctx, S_init, n);
    if (rc) return rc;
    ctx->hook = read_tma_hook();
    ctx->step = 0;
    if (ctx->form == PF_DISCRETE) {
        ctx->scur = 0;
        CK(cudaMemcpy2DAsync(ctx->S[0], ctx->P, S_init, ctx->W, ctx->W, (size_t)ctx->R * ctx->H,
                             cudaMemcpyDeviceToDevice, ctx->st));
        CK(cudaMemsetAsync(ctx->dties, 0, 2 * sizeof(unsigned long long), ctx->st));
        if (ctx->acc && (rc = dca_record(ctx))) return rc;
        rc = run_discrete(ctx, T);
        if (rc) return rc;
        return write_discrete_out(ctx, S_out);
    }
    {
        LaunchScope ls(ctx, K_MISC);
        launch_diff_init(S_init, ctx->H, ctx->W, ctx->P, ctx->work[0], ctx->burn, ctx->st);
    }
    if ((rc = check_launch(ctx, "diff init"))) return rc;
    ctx->cur_ab = ctx->work[0];
    ctx->version++;  // the burnable mask is part of q
    if ((rc = tape_begin(ctx, T))) return rc;
    if ((rc = diff_steps(ctx, T))) return rc;
    return write_diff_out(ctx, S_out);
}

int pf_advance(pf_ctx* ctx, int T, void* S_out) {
    if (!ctx) return fail(nullptr, PF_EINVAL, "pf_advance: ctx is NULL");
    if (T < 0) return fail(ctx, PF_EINVAL, "pf_advance: T must be >= 0");
    ctx->hook = read_tma_hook();
    int rc;
    if (ctx->form == PF_DISCRETE) {
        if ((rc = run_discrete(ctx, T))) return rc;
        return write_discrete_out(ctx, S_out);
    }
    if (!ctx->tape_valid || ctx->t_version != ctx->version) {
        if ((rc = tape_begin(ctx, T))) return rc;
    }
    if ((rc = diff_steps(ctx, T))) return rc;
    return write_diff_out(ctx, S_out);
}

int pf_get_state(pf_ctx* ctx, int* step, void* S) {
    if (!ctx) return fail(nullptr, PF_EINVAL, "pf_get_state: ctx is NULL");
    if (step) *step = ctx->step;
    if (!S) return PF_OK;
    return ctx->form == PF_DISCRETE ? write_discrete_out(ctx, S) : write_diff_out(ctx, S);
}

int pf_set_state(pf_ctx* ctx, int step, const void* S) {
    if (!ctx) return fail(nullptr, PF_EINVAL, "pf_set_state: ctx is NULL");
    if (!S || step < 0) return fail(ctx, PF_EINVAL, "pf_set_state: NULL state or negative step");
    tape_reset(ctx);
    ctx->dca_valid = false;
    ctx->version++;  // a q computed under a reach mask holds for the trajectory it was made on
    if (ctx->form == PF_DISCRETE) {
        int rc = validate_states(ctx, (const uint8_t*)S, (size_t)ctx->R * ctx->H * ctx->W);
        if (rc) return rc;
        CK(cudaMemcpy2DAsync(ctx->S[ctx->scur], ctx->P, S, ctx->W, ctx->W, (size_t)ctx->R * ctx->H,
                             cudaMemcpyDeviceToDevice, ctx->st));
    } else {
        float* dst = (ctx->cur_ab == ctx->work[0]) ? ctx->work[1] : ctx->work[0];
        {
            LaunchScope ls(ctx, K_MISC);
            launch_diff_pack((const float*)S, ctx->H, ctx->W, ctx->P, dst, ctx->st);
        }
        int rc = check_launch(ctx, "diff pack");
        if (rc) return rc;
        ctx->cur_ab = dst;
    }
    ctx->step = step;
    return PF_OK;
}

int pf_stats(pf_ctx* ctx, pf_stats_t* out) {
    if (!ctx || !out) return fail(ctx, PF_EINVAL, "pf_stats: NULL argument");
    CK(cudaMemsetAsync(ctx->dties + 2, 0, 6 * sizeof(unsigned long long), ctx->st));
    {
        LaunchScope ls(ctx, K_MISC);
        if (ctx->form == PF_DISCRETE)
            launch_state_counts(ctx->S[ctx->scur], ctx->R, ctx->H, ctx->W, ctx->P, ctx->dties + 2, ctx->st);
        else
            launch_diff_sums(ctx->cur_ab, ctx->burn, ctx->H, ctx->W, ctx->P, ctx->dties + 2,
                             reinterpret_cast<double*>(ctx->dties + 6), ctx->st);
    }
    int rc = check_launch(ctx, "state statistics");
    if (rc) return rc;
    unsigned long long h[8];
    CK(cudaMemcpyAsync(h, ctx->dties, sizeof(h), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    out->step = ctx->step;
    if (ctx->form == PF_DISCRETE) {
        for (int i = 0; i < 4; ++i) out->cells[i] = (double)h[2 + i];
        out->near_ties_ignite = (long long)h[0];
        out->near_ties_continue = (long long)h[1];
    } else {
        double sa, sb;
        memcpy(&sa, h + 6, sizeof(double));
        memcpy(&sb, h + 7, sizeof(double));
        const double nburn = (double)h[2];
        out->cells[0] = (double)ctx->H * ctx->W - nburn;
        out->cells[1] = nburn - sa;
        out->cells[2] = sb;
        out->cells[3] = sa - sb;
        out->near_ties_ignite = out->near_ties_continue = 0;  // the differentiable form draws nothing
    }
    return PF_OK;
}

int pf_ignition_map(pf_ctx* ctx, float* P_out) {
    if (!ctx || !P_out) return fail(ctx, PF_EINVAL, "pf_ignition_map: NULL argument");
    int rc = ensure_q(ctx, epoch_of(ctx, ctx->step), ctx->step + 1);
    if (rc) return rc;
    {
        LaunchScope ls(ctx, K_MISC);
        if (ctx->form == PF_DISCRETE)
            launch_ignition_map_discrete(dargs(ctx), ctx->S[ctx->scur], ctx->q, P_out, ctx->st);
        else
            launch_ignition_map_diff(ctx->H, ctx->W, ctx->P, ctx->cur_ab, ctx->q, P_out, ctx->st);
    }
    return check_launch(ctx, "ignition map");
}

int pf_backward(pf_ctx* ctx, const float* dL_da_T, const float* dL_db_T, double grad_params[4], float* grad_pveg,
                float* grad_pden) {
    if (!ctx) return fail(nullptr, PF_EINVAL, "pf_backward: ctx is NULL");
    if (!grad_params) return fail(ctx, PF_EINVAL, "pf_backward: grad_params is NULL");
    if (ctx->form != PF_DIFF) return fail(ctx, PF_ESTATE, "pf_backward: only the differentiable form has an adjoint");
    if (!ctx->tape_valid || ctx->t_version != ctx->version)
        return fail(ctx, PF_ESTATE, "pf_backward: no recorded differentiable run (call pf_forward first)");
    const size_t pe = plane_elems(ctx);
    const size_t sbytes = diff_state_bytes(ctx);
    int rc;
    ctx->hook = read_tma_hook();
    // lazily allocated adjoint buffers
    for (int i = 0; i < 2; ++i) {
        if (!ctx->lam[i]) {
            void* p;
            if ((rc = dalloc(ctx, &p, sbytes))) return rc;
            ctx->lam[i] = (float*)p;
        }
        if (!ctx->sig[i]) {
            void* p;
            if ((rc = dalloc(ctx, &p, pe))) return rc;
            ctx->sig[i] = (uint8_t*)p;
        }
    }
    if (!ctx->Gq) {
        void* p;
        if ((rc = dalloc(ctx, &p, 8 * pe * sizeof(float)))) return rc;
        ctx->Gq = (float*)p;
    }
    const int nblk = prep_adjoint_blocks(ctx->H, ctx->W);
    if (!ctx->partials) {
        void* p;
        if ((rc = dalloc(ctx, &p, (size_t)nblk * 4 * sizeof(double) + 4 * sizeof(double)))) return rc;
        ctx->partials = (double*)p;
        ctx->gacc = ctx->partials + (size_t)nblk * 4;
    }
    const int segmax = ctx->K > 1 ? ctx->K : 0;  // states s0 .. s0+K-1 of one segment, consecutive
    if (ctx->seg_cap < segmax) {
        if (ctx->seg_buf) dfree(ctx, ctx->seg_buf);
        ctx->seg_buf = nullptr;
        ctx->seg_cap = 0;
        void* p;
        if ((rc = dalloc(ctx, &p, sbytes * (size_t)segmax))) return rc;
        ctx->seg_buf = (float*)p;
        ctx->seg_cap = segmax;
        ctx->seg_halo = 0;  // contents unknown: cleared before the first blocked recompute
    }
    const size_t selems = 2 * pe;
    const int kern = choose_kernel(ctx);
    CUtensorMap tseg;
    const bool adj_blocked = kern == 2 && ctx->seg_buf && adjoint_blocked_configure() == 0 &&
                             encode_f32_3d(&tseg, ctx->seg_buf, ctx->P, ctx->H, 2 * ctx->seg_cap,
                                           diff_blocked_box_cols(), diff_blocked_box_rows(), 2);
    cudaGetLastError();
    // terminal adjoint, in the scaled form (exponents from the state at T)
    {
        LaunchScope ls(ctx, K_MISC);
        launch_adjoint_init(dL_da_T, dL_db_T, ctx->cur_ab, ctx->H, ctx->W, ctx->P, ctx->lam[0], ctx->sig[0], ctx->st);
    }
    if ((rc = check_launch(ctx, "adjoint init"))) return rc;
    CK(cudaMemsetAsync(ctx->gacc, 0, 4 * sizeof(double), ctx->st));
    const size_t cell_bytes = (size_t)ctx->H * ctx->W * sizeof(float);
    if (grad_pveg) CK(cudaMemsetAsync(grad_pveg, 0, cell_bytes, ctx->st));
    if (grad_pden) CK(cudaMemsetAsync(grad_pden, 0, cell_bytes, ctx->st));
    CK(cudaMemsetAsync(ctx->Gq, 0, 8 * pe * sizeof(float), ctx->st));
    const size_t ntiles_adj = (size_t)adjoint_blocked_tiles(ctx->H, ctx->P);
    CK(cudaMemsetAsync(ctx->adeadcnt, 0, ntiles_adj, ctx->st));
    CK(cudaMemsetAsync(ctx->gqdirty, 0, ntiles_adj, ctx->st));

    const int T_end = ctx->step;
    int lcur = 0;
    int cur_e = -1;
    // the blocked adjoint's pre-passes mark the tiles that may add to dL/dq; a plain
    // adjoint step may add anywhere
    bool gq_anywhere = false;
    auto flush = [&](int e) -> int {
        {
            LaunchScope ls(ctx, K_PADJ);
            PrepArgs g = prep_args(ctx, e, true);
            if (!gq_anywhere) {
                g.gq_dirty = ctx->gqdirty;
                g.gq_tiles_x = (ctx->P + 47) / 48;
            }
            launch_prep_adjoint(g, ctx->Gq, ctx->partials, grad_pveg, grad_pden, ctx->st);
        }
        int r = check_launch(ctx, "prep adjoint");
        if (r) return r;
        CK(cudaMemsetAsync(ctx->gqdirty, 0, ntiles_adj, ctx->st));
        gq_anywhere = false;
        {
            LaunchScope ls(ctx, K_RED);
            launch_reduce_partials(ctx->partials, nblk, ctx->gacc, ctx->st);
        }
        return check_launch(ctx, "fp64 reduction");  // prep_adjoint left Gq zeroed
    };
    // switch q (and the dL/dq accumulator) to the epoch of step t
    auto enter_epoch = [&](int t) -> int {
        const int e = epoch_of(ctx, t);
        if (e == cur_e) return PF_OK;
        int r;
        if (cur_e >= 0 && (r = flush(cur_e))) return r;
        cur_e = e;
        if (e < (int)ctx->qcache.size() && ctx->qcache[e] && ctx->qcache_ver[e] == ctx->t_version) {
            // the taped forward's q of this epoch (same parameters, fields and wind)
            if ((r = use_q_buffer(ctx, ctx->qcache[e]))) return r;
        } else {
            if ((r = use_q_buffer(ctx, ctx->q_own))) return r;
            {
                LaunchScope ls(ctx, K_PREP);
                PrepArgs g = prep_args(ctx, e, true);
                // the blocks the taped forward computed (the rest of the buffer keeps
                // finite q values nothing reads), else every cell
                if (e < (int)ctx->qmask_state.size() && ctx->qmask_state[e] == 1 && ctx->qmasks) {
                    g.reach = ctx->qmasks + (size_t)e * prep_reach_bytes(ctx->H, ctx->W);
                    g.reach_bw = (ctx->W + 31) / 32;
                }
                launch_prep(g, ctx->q, ctx->st);
            }
            if ((r = check_launch(ctx, "prep"))) return r;
        }
        ctx->q_key_epoch = -1;  // q now holds the recorded parameters' q
        return PF_OK;
    };
    const float pc = ctx->t_pc;
    // adjoint steps t = t1-1 .. t0 over states held consecutively in `buf` (state
    // index z(t) = t - tbase), with its tensor map
    // With `align` > 0 the launches are [t0 + align i, t0 + align (i + 1)) like the
    // segment's recompute launches, whose recorded tile flags then describe exactly the
    // states of each adjoint launch (kFrozen tiles read one state for all steps).
    // first / tmap0 (nullable): the state at tbase when it is not in buf (a checkpoint)
    auto adjoint_run = [&](const float* buf, const CUtensorMap* tmap, int tbase, int t0, int t1, int align = 0,
                           const float* first = nullptr, const CUtensorMap* tmap0 = nullptr) -> int {
        auto state_at = [&](int t) { return (t == tbase && first) ? first : buf + (size_t)(t - tbase) * selems; };
        int r;
        while (t1 > t0) {
            if (tmap) {
                int n = std::min(adjoint_blocked_max_steps(), t1 - t0);
                if (align > 0) n = (t1 - t0) % align ? (t1 - t0) % align : align;
                // the earliest recorded activity at or after t1 - 1, if any
                int ri = -1;
                for (int k = 0; k < (int)ctx->actrec_end.size(); ++k)
                    if (ctx->actrec_end[k] >= t1 - 1 && (ri < 0 || ctx->actrec_end[k] < ctx->actrec_end[ri])) ri = k;
                {
                    LaunchScope ls(ctx, K_ATILES);
                    if (ri >= 0)
                        launch_adjoint_tiles_flags(ctx->actrec + (size_t)ri * diff_blocked_tiles(8, ctx->H, ctx->P),
                                                   ctx->H, ctx->W, ctx->P, n, ctx->lam[1 - lcur], ctx->sig[1 - lcur],
                                                   ctx->adeadcnt, ctx->tile_list, ctx->dflags + 8,
                                                   // aligned: the record is this launch's own recompute
                                                   // (a one-step launch reads one state anyway)
                                                   align > 0, ctx->gqdirty,
                                                   ctx->dskip + K_ABLK, ctx->dskip + K_ATILES, ctx->st);
                    else
                        launch_adjoint_tiles(state_at(t1 - 1), ctx->H, ctx->W, ctx->P, n,
                                             ctx->lam[1 - lcur], ctx->sig[1 - lcur], ctx->tile_list, ctx->dflags + 8,
                                             ctx->gqdirty, ctx->dskip + K_ABLK, ctx->st);
                }
                // the live tiles, then the frozen ones (a kernel of their own)
                CUtensorMap tlam;
                if (!encode_f32_3d(&tlam, ctx->lam[lcur], ctx->P, ctx->H, 2, diff_blocked_box_cols(),
                                   diff_blocked_box_rows(), 2))
                    return fail(ctx, PF_ECUDA, "tensor map encoding of lambda failed");
                for (int fz = 0; fz < 2; ++fz) {
                    LaunchScope ls(ctx, fz ? K_AFRZ : K_ABLK, n);
                    launch_adjoint_blocked(tmap, tmap0 ? tmap0 : tmap, &ctx->tmapQ, &tlam, ctx->H, ctx->P, pc,
                                           t1 - 1 - tbase, n, ctx->lam[lcur], ctx->sig[lcur], ctx->lam[1 - lcur],
                                           ctx->sig[1 - lcur], ctx->Gq, ctx->tile_list, ctx->dflags + 8, ctx->nsm,
                                           ctx->dflags, ctx->hook, fz != 0, ctx->st);
                }
                if ((r = check_launch(ctx, "adjoint blocked"))) return r;
                t1 -= n;
            } else {
                gq_anywhere = true;
                {
                    LaunchScope ls(ctx, K_ADJ);
                    launch_adjoint_step(ctx->H, ctx->W, ctx->P, pc, state_at(t1 - 1), ctx->q,
                                        ctx->lam[lcur], ctx->sig[lcur], ctx->lam[1 - lcur], ctx->sig[1 - lcur],
                                        ctx->Gq, ctx->st);
                }
                if ((r = check_launch(ctx, "adjoint step"))) return r;
                t1 -= 1;
            }
            lcur = 1 - lcur;
        }
        return PF_OK;
    };
    if (ctx->K == 1) {
        // every state is on the tape: no recomputation; runs end at wind-epoch starts
        CUtensorMap tarena;
        const bool ok = kern == 2 && adjoint_blocked_configure() == 0 &&
                        encode_f32_3d(&tarena, ctx->arena, ctx->P, ctx->H, 2 * ctx->arena_cap,
                                      diff_blocked_box_cols(), diff_blocked_box_rows(), 2);
        cudaGetLastError();
        const int t_start = ctx->tape_start;
        for (int t1 = T_end; t1 > t_start;) {
            if ((rc = enter_epoch(t1 - 1))) return rc;
            const int t0 = std::max(t_start, ctx->winds[cur_e].from);
            if ((rc = adjoint_run(ctx->arena, ok ? &tarena : nullptr, t_start, t0, t1))) return rc;
            t1 = t0;
        }
    } else {
        // recompute and adjoint launches of `chunk` steps from each segment start, so that
        // the recorded flags of a recompute launch describe an adjoint launch's states
        const int chunk = std::min(blocked_k(ctx), adjoint_blocked_max_steps());
        const bool aligned = kern == 2 && adj_blocked && blocked_k(ctx) > 4;
        // the tile tape's records, by first step (only complete ones: every block fitted)
        std::vector<int> rec_at;
        if (kern == 2 && ctx->ttape_on && !ctx->ttape_rec.empty()) {
            const size_t nr = ctx->ttape_rec.size();
            ctx->ttape_meta_h.assign(4 * nr, 0ull);
            CK(cudaMemcpyAsync(ctx->ttape_meta_h.data(), ctx->ttape_meta, 4 * nr * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, ctx->st));
            CK(cudaMemsetAsync(ctx->dflags + 14, 0, sizeof(int), ctx->st));
            CK(cudaStreamSynchronize(ctx->st));
            rec_at.assign((size_t)(T_end - ctx->tape_start + 1), -1);
            ctx->ttape_need = 0;
            ctx->ttape_need_blk = ctx->ttape_blk;
            ctx->ttape_short = false;
            for (size_t L = 0; L < nr; ++L) {
                const int t0 = ctx->ttape_rec[L].first - ctx->tape_start;
                ctx->ttape_need += ctx->ttape_meta_h[4 * L + 1] * ctx->ttape_meta_h[4 * L + 2];
                if (!ctx->ttape_meta_h[4 * L + 3]) ctx->ttape_short = true;
                if (ctx->ttape_meta_h[4 * L + 3] && t0 >= 0 && t0 < (int)rec_at.size()) rec_at[t0] = (int)L;
            }
        }
        for (int si = (int)ctx->ckpts.size() - 1; si >= 0; --si) {
            const int s0 = ctx->ckpts[si].first;
            const int s1 = (si + 1 < (int)ctx->ckpts.size()) ? ctx->ckpts[si + 1].first : T_end;
            if (s1 <= s0) continue;
            if ((rc = enter_epoch(s0))) return rc;
            // the segment's states s0 .. s1-1: the checkpoint itself, then the recomputed
            // ones in slots 1.. of the segment buffer (slot 0 unused)
            float* seg = ctx->seg_buf;
            if (kern == 2) {
                // blocked recompute: the slots hold zeros outside each tile's seg_rng range
                const int halo = blocked_k(ctx) <= 4 ? 4 : 8;
                if (ctx->seg_halo != halo) {
                    const size_t nt = (size_t)std::max(diff_blocked_tiles(8, ctx->H, ctx->P),
                                                       diff_blocked_tiles(4, ctx->H, ctx->P));
                    if (!ctx->seg_rng) {
                        void* p;
                        if ((rc = dalloc(ctx, &p, nt * sizeof(uint32_t)))) return rc;
                        ctx->seg_rng = (uint32_t*)p;
                    }
                    CK(cudaMemsetAsync(seg, 0, sbytes * (size_t)ctx->seg_cap, ctx->st));
                    CK(cudaMemsetAsync(ctx->seg_rng, 0, nt * sizeof(uint32_t), ctx->st));
                    ctx->seg_halo = halo;
                }
            } else {
                ctx->seg_halo = 0;  // the plain kernel writes every cell of the slots
            }
            const float* ck = slot_ptr(ctx, ctx->ckpts[si].second);
            ctx->seg_slot0 = ck;
            CUtensorMap tck;
            if (adj_blocked && !encode_f32_3d(&tck, ck, ctx->P, ctx->H, 2, diff_blocked_box_cols(),
                                              diff_blocked_box_rows(), 2))
                return fail(ctx, PF_ECUDA, "tensor map encoding of a checkpoint failed");
            // the segment's states, recomputed or (use_tape) copied from the tile tape where
            // a complete record covers a launch; returns whether any launch used the tape
            auto run_segment = [&](bool use_tape, bool* used_tape) -> int {
                *used_tape = false;
                ctx->fl_state = nullptr;  // a new chain starts from the checkpoint, with its recorded flags if any
                {
                    const int cs = ctx->ckpts[si].second;
                    const bool rec = cs < (int)ctx->ckact_halo.size() && ctx->ckact_halo[cs] != 0;
                    const size_t nt = (size_t)std::max(diff_blocked_tiles(8, ctx->H, ctx->P),
                                                       diff_blocked_tiles(4, ctx->H, ctx->P));
                    ctx->fl_seed = rec ? ctx->ckact + nt * cs : nullptr;
                    ctx->fl_seed_halo = rec ? ctx->ckact_halo[cs] : 0;
                }
                ctx->actrec_end.clear();
                ctx->actrec_on = true;
                int r;
                for (int t = s0; t < s1 - 1;) {
                    const float* in = t == s0 ? ck : seg + (size_t)(t - s0) * selems;
                    float* nxt = seg + (size_t)(t - s0 + 1) * selems;
                    if (kern == 2) {
                        // launches of `chunk` steps from s0, the adjoint's launches below
                        const int n = std::min(chunk, s1 - 1 - t);
                        int L = -1;
                        if (use_tape && t - ctx->tape_start < (int)rec_at.size()) {
                            L = rec_at[(size_t)(t - ctx->tape_start)];
                            if (L >= 0 && (int)ctx->ttape_meta_h[4 * (size_t)L + 1] < n) L = -1;
                        }
                        if (L >= 0) *used_tape = true;
                        if ((r = diff_blocked_launch(ctx, in, pc, n, nullptr, nxt, true, t + n, aligned, nullptr, -1,
                                                     L)))
                            return r;
                        t += n;
                    } else {
                        {
                            LaunchScope ls(ctx, K_FSTEP);
                            launch_diff_step(ctx->H, ctx->W, ctx->P, pc, in, nxt, ctx->q, ctx->st);
                        }
                        if ((r = check_launch(ctx, "diff step (recompute)"))) return r;
                        t += 1;
                    }
                }
                return PF_OK;
            };
            bool used_tape = false;
            if ((rc = run_segment(!rec_at.empty(), &used_tape))) return rc;
            if (used_tape) {
                // a listed tile the tape's record lacks (its launch was listed differently):
                // recompute the segment
                CK(cudaMemcpyAsync(ctx->hflags + 14, ctx->dflags + 14, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
                CK(cudaStreamSynchronize(ctx->st));
                if (ctx->hflags[14] != 0) {
                    CK(cudaMemsetAsync(ctx->dflags + 14, 0, sizeof(int), ctx->st));
                    if ((rc = run_segment(false, &used_tape))) return rc;
                }
            }
            if ((rc = adjoint_run(seg, adj_blocked ? &tseg : nullptr, s0, s0, s1, aligned ? chunk : 0, ck,
                                  adj_blocked ? &tck : nullptr)))
                return rc;
        }
    }
    ctx->fl_seed = nullptr;
    if (cur_e >= 0 && (rc = flush(cur_e))) return rc;
    CK(cudaMemcpyAsync(ctx->hflags + 4, ctx->gacc, 4 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    if ((rc = device_error(ctx))) return rc;  // synchronises the stream
    memcpy(grad_params, ctx->hflags + 4, 4 * sizeof(double));
    return PF_OK;
}

int pf_profile_read(pf_ctx* ctx, int max_kinds, const char** kinds, long long* launches, long long* cell_steps,
                    long long* skipped_cell_steps, double* ms, int reset) {
    if (!ctx) return fail(nullptr, PF_EINVAL, "pf_profile_read: ctx is NULL");
    unsigned long long skip[K_NKINDS];
    CK(cudaMemcpyAsync(skip, ctx->dskip, sizeof(skip), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    prof_collect(ctx);
    int n = std::min(max_kinds, (int)K_NKINDS);
    for (int i = 0; i < n; ++i) {
        if (kinds) kinds[i] = kKindNames[i];
        if (launches) launches[i] = ctx->launches[i];
        if (cell_steps) cell_steps[i] = ctx->cell_steps[i];
        if (skipped_cell_steps) skipped_cell_steps[i] = (long long)skip[i];
        if (ms) ms[i] = ctx->prof_ms[i];
    }
    if (reset) {
        for (int i = 0; i < K_NKINDS; ++i) {
            ctx->launches[i] = 0;
            ctx->cell_steps[i] = 0;
            ctx->prof_ms[i] = 0.0;
        }
        CK(cudaMemsetAsync(ctx->dskip, 0, sizeof(skip), ctx->st));
    }
    return n;
}

int pf_set_accumulator(pf_ctx* ctx, float* acc) {
    if (!ctx) return fail(nullptr, PF_EINVAL, "pf_set_accumulator: ctx is NULL");
    if (ctx->form != PF_DISCRETE) return fail(ctx, PF_EINVAL, "pf_set_accumulator: the accumulator is of the discrete form");
    ctx->acc = acc;
    ctx->dca_valid = false;
    return PF_OK;
}

int pf_reseed(pf_ctx* ctx, uint64_t seed) {
    if (!ctx) return fail(nullptr, PF_EINVAL, "pf_reseed: ctx is NULL");
    ctx->seed = seed;
    ctx->dca_valid = false;
    tape_reset(ctx);
    return PF_OK;
}

int pf_backward_dca(pf_ctx* ctx, const float* dL_dacc, const uint8_t* step_mask, double grad_params[4],
                    float* grad_pveg, float* grad_pden) {
    if (!ctx) return fail(nullptr, PF_EINVAL, "pf_backward_dca: ctx is NULL");
    if (!dL_dacc || !grad_params) return fail(ctx, PF_EINVAL, "pf_backward_dca: NULL dL_dacc or grad_params");
    if (ctx->form != PF_DISCRETE || !ctx->dca_valid)
        return fail(ctx, PF_ESTATE, "pf_backward_dca: no trajectory recorded (set an accumulator, then pf_forward)");
    if (ctx->dca_version != ctx->version)
        return fail(ctx, PF_ESTATE, "pf_backward_dca: parameters, fields or wind changed since pf_forward");
    const size_t pe = plane_elems(ctx);
    const size_t sb = (size_t)ctx->R * pe;
    int rc;
    if (!ctx->Gq) {
        void* p;
        if ((rc = dalloc(ctx, &p, 8 * pe * sizeof(float)))) return rc;
        ctx->Gq = (float*)p;
    }
    const int nblk = prep_adjoint_blocks(ctx->H, ctx->W);
    if (!ctx->partials) {
        void* p;
        if ((rc = dalloc(ctx, &p, (size_t)nblk * 4 * sizeof(double) + 4 * sizeof(double)))) return rc;
        ctx->partials = (double*)p;
        ctx->gacc = ctx->partials + (size_t)nblk * 4;
    }
    const size_t cell_bytes = (size_t)ctx->H * ctx->W * sizeof(float);
    CK(cudaMemsetAsync(ctx->gacc, 0, 4 * sizeof(double), ctx->st));
    if (grad_pveg) CK(cudaMemsetAsync(grad_pveg, 0, cell_bytes, ctx->st));
    if (grad_pden) CK(cudaMemsetAsync(grad_pden, 0, cell_bytes, ctx->st));
    CK(cudaMemsetAsync(ctx->Gq, 0, 8 * pe * sizeof(float), ctx->st));
    CK(cudaMemcpyAsync(ctx->dca_S[0], ctx->dca_S0, sb, cudaMemcpyDeviceToDevice, ctx->st));
    DiscreteArgs g = dargs(ctx);
    g.p_continue = ctx->t_pc;
    g.acc = nullptr;
    g.ties = nullptr;  // a replay: its draws were counted when the trajectory was made
    auto flush = [&](int e) -> int {
        {
            LaunchScope ls(ctx, K_PADJ);
            launch_prep_adjoint(prep_args(ctx, e, true), ctx->Gq, ctx->partials, grad_pveg, grad_pden, ctx->st);
        }
        int r = check_launch(ctx, "prep adjoint");
        if (r) return r;
        {
            LaunchScope ls(ctx, K_RED);
            launch_reduce_partials(ctx->partials, nblk, ctx->gacc, ctx->st);
        }
        return check_launch(ctx, "fp64 reduction");  // prep_adjoint left Gq zeroed
    };
    // replay the trajectory (same Philox counters) with the plain step; at every attached
    // step add the gradient of the cells that ignite in it
    int cur = 0, cur_e = -1;
    for (int t = 0; t < ctx->step; ++t) {
        const int e = epoch_of(ctx, t);
        if (e != cur_e) {
            if (cur_e >= 0 && (rc = flush(cur_e))) return rc;
            cur_e = e;
            {
                LaunchScope ls(ctx, K_PREP);
                launch_prep(prep_args(ctx, e, true), ctx->q, ctx->st);
            }
            if ((rc = check_launch(ctx, "prep"))) return rc;
            ctx->q_key_epoch = -1;
        }
        {
            LaunchScope ls(ctx, K_DSTEP);
            launch_discrete_step(g, ctx->dca_S[cur], ctx->dca_S[1 - cur], ctx->q, (uint32_t)t, ctx->st);
        }
        if ((rc = check_launch(ctx, "discrete step (replay)"))) return rc;
        if (!step_mask || step_mask[t]) {
            {
                LaunchScope ls(ctx, K_DCA);
                launch_dca_step(g, ctx->dca_S[cur], ctx->dca_S[1 - cur], ctx->q, dL_dacc, ctx->Gq, ctx->st);
            }
            if ((rc = check_launch(ctx, "dca step"))) return rc;
        }
        cur = 1 - cur;
    }
    ctx->fl_seed = nullptr;
    if (cur_e >= 0 && (rc = flush(cur_e))) return rc;
    CK(cudaMemcpyAsync(ctx->hflags + 4, ctx->gacc, 4 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    std::memcpy(grad_params, ctx->hflags + 4, 4 * sizeof(double));
    return PF_OK;
}

int pf_arrival_probability(const uint8_t* S, int R, int H, int W, float* P_out, void* cuda_stream) {
    if (!S || !P_out || R < 1 || H < 1 || W < 1) return fail(nullptr, PF_EINVAL, "pf_arrival_probability: bad arguments");
    launch_arrival(S, R, (int64_t)H * W, P_out, (cudaStream_t)cuda_stream);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, PF_ECUDA, "pf_arrival_probability: %s", cudaGetErrorString(e));
    return PF_OK;
}

// device scratch of the counting entry points: one small buffer per thread
static unsigned long long* count_scratch(int n, int* rc) {
    static thread_local unsigned long long* buf = nullptr;
    static thread_local int cap = 0;
    *rc = PF_OK;
    if (cap < n) {
        if (buf) cudaFree(buf);
        buf = nullptr;
        cap = 0;
        if (cudaMalloc((void**)&buf, sizeof(unsigned long long) * (size_t)n) != cudaSuccess) {
            cudaGetLastError();
            *rc = PF_ENOMEM;
            return nullptr;
        }
        cap = n;
    }
    return buf;
}

int pf_affected_count(const uint8_t* S, int R, int64_t HW, long long* counts, void* cuda_stream) {
    if (!S || !counts || R < 1 || HW < 1) return fail(nullptr, PF_EINVAL, "pf_affected_count: bad arguments");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int rc;
    unsigned long long* d = count_scratch(R, &rc);
    if (!d) return fail(nullptr, rc, "pf_affected_count: scratch allocation failed");
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long) * R, st);
    if (e == cudaSuccess) {
        launch_count(S, nullptr, HW, R, d, st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts, d, sizeof(long long) * R, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(nullptr, PF_ECUDA, "pf_affected_count: %s", cudaGetErrorString(e));
    return PF_OK;
}

int pf_manhattan(const uint8_t* SA, const uint8_t* SB, int T, int64_t HW, long long* out, void* cuda_stream) {
    if (!SA || !SB || !out || T < 1 || HW < 1) return fail(nullptr, PF_EINVAL, "pf_manhattan: bad arguments");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int rc;
    unsigned long long* d = count_scratch(2 * T + 1, &rc);
    if (!d) return fail(nullptr, rc, "pf_manhattan: scratch allocation failed");
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long) * (2 * (size_t)T + 1), st);
    if (e == cudaSuccess) {
        launch_count(SA, nullptr, HW, T, d, st);
        launch_count(SB, nullptr, HW, T, d + T, st);
        launch_l1(d, d + T, T, d + 2 * T, st);
        e = cudaGetLastError();
    }
    unsigned long long h = 0ull;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d + 2 * T, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(nullptr, PF_ECUDA, "pf_manhattan: %s", cudaGetErrorString(e));
    *out = (long long)h;
    return PF_OK;
}

int pf_jaccard(const uint8_t* A, const uint8_t* B, int64_t n, double* out, void* cuda_stream) {
    if (!A || !B || !out || n < 1) return fail(nullptr, PF_EINVAL, "pf_jaccard: bad arguments");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int rc;
    unsigned long long* d = count_scratch(2, &rc);
    if (!d) return fail(nullptr, rc, "pf_jaccard: scratch allocation failed");
    unsigned long long h[2] = {0, 0};
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(h), st);
    if (e == cudaSuccess) {
        launch_count(A, B, n, 1, d, st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(nullptr, PF_ECUDA, "pf_jaccard: %s", cudaGetErrorString(e));
    *out = h[1] ? (double)h[0] / (double)h[1] : 1.0;
    return PF_OK;
}

int pf_loss_eq10(const float* yhat, const float* y, int H, int W, float* dL_dyhat, double* loss, void* cuda_stream) {
    if (!yhat || !y || H < 1 || W < 1) return fail(nullptr, PF_EINVAL, "pf_loss_eq10: NULL map or empty grid");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int nblk = eq10_blocks(H, W);
    static thread_local double* cached = nullptr;
    static thread_local size_t cached_bytes = 0;
    const size_t need = eq10_scratch_bytes(H, W);
    if (cached_bytes < need) {
        if (cached) cudaFree(cached);
        if (cudaMalloc((void**)&cached, need) != cudaSuccess) {
            cudaGetLastError();
            cached = nullptr;
            cached_bytes = 0;
            return fail(nullptr, PF_ENOMEM, "pf_loss_eq10: scratch allocation failed");
        }
        cached_bytes = need;
    }
    launch_eq10(yhat, y, H, W, dL_dyhat, cached, nblk, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && loss) {
        double h = 0.0;
        e = cudaMemcpyAsync(&h, eq10_result(cached, nblk), sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        *loss = h;
    }
    if (e != cudaSuccess) return fail(nullptr, PF_ECUDA, "pf_loss_eq10: %s", cudaGetErrorString(e));
    return PF_OK;
}

int pf_loss_bce(const float* a, const float* y, int64_t n, float* dL_da, double* loss, void* cuda_stream) {
    if (!a || !y || n <= 0) return fail(nullptr, PF_EINVAL, "pf_loss_bce: NULL input or n <= 0");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int nblk = bce_blocks(n);
    double* partials = nullptr;
    static thread_local double* cached = nullptr;
    static thread_local int cached_n = 0;
    if (cached_n < nblk + 1) {
        if (cached) cudaFree(cached);
        if (cudaMalloc((void**)&cached, sizeof(double) * (nblk + 1)) != cudaSuccess) {
            cudaGetLastError();
            cached = nullptr;
            cached_n = 0;
            return fail(nullptr, PF_ENOMEM, "pf_loss_bce: scratch allocation failed");
        }
        cached_n = nblk + 1;
    }
    partials = cached;
    launch_bce(a, y, n, dL_da, partials, nblk, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, PF_ECUDA, "pf_loss_bce: %s", cudaGetErrorString(e));
    if (loss) {
        double h = 0.0;
        e = cudaMemcpyAsync(&h, partials + nblk, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(nullptr, PF_ECUDA, "pf_loss_bce: %s", cudaGetErrorString(e));
        *loss = h;
    }
    return PF_OK;
}

// One submission (a wave) of jobs that were validated by pf_batch_submit: one arena,
// one captured graph, one persistent forward kernel and one adjoint kernel.
// statistics of this thread's last pf_batch_submit, summed over its waves
thread_local pf_batch_stats_t g_batch_stats{};

static int batch_submit_wave(const pf_job* jobs, int n, cudaStream_t st) {
    pf_ctx* ctx = nullptr;  // context-free: errors go to pf_last_error(NULL)
    const int kB = batch_steps_per_item(), kTR = batch_tile_rows(), kTC = batch_tile_cols();
    // order jobs by block count, descending (block-major item order)
    std::vector<int> order(n);
    std::vector<int> nblk(n);
    for (int i = 0; i < n; ++i) {
        order[i] = i;
        nblk[i] = std::max(1, (jobs[i].T + kB - 1) / kB);
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return nblk[x] > nblk[y]; });
    // one arena: per job two state buffers, q, a burnable mask and tile counters
    struct Lay {
        size_t st, q, mask, gen, stbytes;
        int P, tx, ty;
        bool adj;  // differentiable job with an adjoint
        size_t tape, lam, sig, gq, genb;
        int btx, bty;
    };
    const int kAR = batch_adj_tile_rows(), kAC = batch_adj_tile_cols();
    std::vector<Lay> lay(n);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
    for (int k = 0; k < n; ++k) {
        const pf_job& J = jobs[order[k]];
        Lay& L = lay[k];
        L.P = pitch_of(J.W);
        L.tx = (J.W + kTC - 1) / kTC;
        L.ty = (J.H + kTR - 1) / kTR;
        const size_t plane = (size_t)J.H * L.P;
        L.stbytes = J.form == PF_DISCRETE ? plane : 2 * plane * sizeof(float);
        L.st = take(2 * L.stbytes);
        L.q = take(8 * plane * sizeof(float));
        L.mask = take((size_t)J.H * J.W);
        L.gen = take((size_t)L.tx * L.ty * sizeof(int));
        L.adj = J.dL_da != nullptr;
        if (L.adj) {
            L.btx = (J.W + kAC - 1) / kAC;
            L.bty = (J.H + kAR - 1) / kAR;
            L.tape = take((size_t)(J.T + 1) * 2 * plane * sizeof(float));
            L.lam = take(2 * 2 * plane * sizeof(float));
            L.sig = take(2 * plane);
            L.gq = take(8 * plane * sizeof(float));
            L.genb = take((size_t)L.btx * L.bty * sizeof(int));
        }
    }
    // backward: the adjoint jobs in the same (block count, descending) order
    std::vector<int> ab;  // positions in `order`
    for (int k = 0; k < n; ++k)
        if (lay[k].adj) ab.push_back(k);
    const int nb = (int)ab.size();
    const int max_blk_b = nb ? nblk[order[ab[0]]] : 0;
    std::vector<long long> tile_pref_b(nb + 1, 0), blk_start_b(max_blk_b + 1, 0);
    std::vector<int> jobs_in_blk_b(std::max(1, max_blk_b), 0);
    for (int k = 0; k < nb; ++k) tile_pref_b[k + 1] = tile_pref_b[k] + (long long)lay[ab[k]].btx * lay[ab[k]].bty;
    for (int b = 0; b < max_blk_b; ++b) {
        int m = 0;
        while (m < nb && nblk[order[ab[m]]] > b) ++m;
        jobs_in_blk_b[b] = m;
        blk_start_b[b + 1] = blk_start_b[b] + tile_pref_b[m];
    }
    int nblk_prep = 1;
    for (int k : ab) nblk_prep = std::max(nblk_prep, prep_adjoint_blocks(jobs[order[k]].H, jobs[order[k]].W));
    const int max_blk = nblk[order[0]];
    std::vector<long long> tile_pref(n + 1, 0), blk_start(max_blk + 1, 0);
    std::vector<int> jobs_in_blk(max_blk, 0);
    for (int k = 0; k < n; ++k) tile_pref[k + 1] = tile_pref[k] + (long long)lay[k].tx * lay[k].ty;
    for (int b = 0; b < max_blk; ++b) {
        int m = 0;
        while (m < n && nblk[order[m]] > b) ++m;
        jobs_in_blk[b] = m;
        blk_start[b + 1] = blk_start[b] + tile_pref[m];
    }
    const size_t o_jobs = take(sizeof(BatchJobDev) * n);
    const size_t o_bs = take(sizeof(long long) * (max_blk + 1));
    const size_t o_tp = take(sizeof(long long) * (n + 1));
    const size_t o_jb = take(sizeof(int) * max_blk);
    const size_t o_ctl = take(sizeof(unsigned long long) + sizeof(int) * 4);
    const size_t o_vf = take(sizeof(int) * n);  // per-job input validation flags
    const size_t o_jobs_b = take(sizeof(BatchJobDev) * std::max(1, nb));
    const size_t o_bs_b = take(sizeof(long long) * (max_blk_b + 1));
    const size_t o_tp_b = take(sizeof(long long) * (nb + 1));
    const size_t o_jb_b = take(sizeof(int) * std::max(1, max_blk_b));
    const size_t o_ctl_b = take(sizeof(unsigned long long));
    const size_t o_part = take(sizeof(double) * 4 * (size_t)nblk_prep);
    const size_t o_stats = take(sizeof(unsigned long long) * kStatCount);
    char* arena = nullptr;
    if (cudaMalloc((void**)&arena, off) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, PF_ENOMEM, "pf_batch_submit: %zu-byte arena allocation failed", off);
    }
    std::vector<BatchJobDev> hj(n);
    for (int k = 0; k < n; ++k) {
        const pf_job& J = jobs[order[k]];
        const Lay& L = lay[k];
        BatchJobDev& D = hj[k];
        D.H = J.H; D.W = J.W; D.P = L.P; D.T = J.T; D.form = J.form; D.nblk = nblk[order[k]];
        D.tiles_x = L.tx; D.tiles_y = L.ty;
        D.key0 = (uint32_t)J.seed; D.key1 = (uint32_t)(J.seed >> 32); D.run = J.run; D.fire = J.fire_id;
        D.pc = J.p_continue;
        D.st[0] = arena + L.st;
        D.st[1] = arena + L.st + L.stbytes;
        D.q = (const float*)(arena + L.q);
        D.gen = (int*)(arena + L.gen);
        D.out = J.S_out;
        D.tape = nullptr;
        D.lam[0] = D.lam[1] = nullptr;
        D.sig[0] = D.sig[1] = nullptr;
        D.Gq = nullptr;
        D.gen_b = nullptr;
        D.btiles_x = D.btiles_y = 0;
        if (L.adj) {
            const size_t plane = (size_t)J.H * L.P;
            D.tape = (float*)(arena + L.tape);
            D.lam[0] = (float*)(arena + L.lam);
            D.lam[1] = D.lam[0] + 2 * plane;
            D.sig[0] = (uint8_t*)(arena + L.sig);
            D.sig[1] = D.sig[0] + plane;
            D.Gq = (float*)(arena + L.gq);
            D.gen_b = (int*)(arena + L.genb);
            D.btiles_x = L.btx;
            D.btiles_y = L.bty;
        }
    }
    std::vector<BatchJobDev> hjb(std::max(1, nb));
    for (int k = 0; k < nb; ++k) hjb[k] = hj[ab[k]];
    unsigned long long* counter = (unsigned long long*)(arena + o_ctl);
    int* derr = (int*)(arena + o_ctl + sizeof(unsigned long long));
    int rc = PF_OK;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaSuccess;
    const char* sl = getenv("PF_BATCH_WAIT_NS");
    const char* wh = getenv("PF_BATCH_TEST_WITHHOLD");
    BatchPlan plan;
    plan.jobs = (const BatchJobDev*)(arena + o_jobs);
    plan.blk_start = (const long long*)(arena + o_bs);
    plan.tile_pref = (const long long*)(arena + o_tp);
    plan.jobs_in_blk = (const int*)(arena + o_jb);
    plan.max_blk = max_blk;
    plan.total = blk_start[max_blk];
    plan.counter = counter;
    plan.err = derr;
    plan.wait_limit_ns = sl ? std::max(1000ll, atoll(sl)) : 4000000000ll;  // 4 s
    plan.withhold = wh ? atoi(wh) : 0;
    plan.stats = (unsigned long long*)(arena + o_stats);
    BatchPlan plan_b = plan;
    plan_b.jobs = (const BatchJobDev*)(arena + o_jobs_b);
    plan_b.blk_start = (const long long*)(arena + o_bs_b);
    plan_b.tile_pref = (const long long*)(arena + o_tp_b);
    plan_b.jobs_in_blk = (const int*)(arena + o_jb_b);
    plan_b.max_blk = max_blk_b;
    plan_b.total = blk_start_b[max_blk_b];
    plan_b.counter = (unsigned long long*)(arena + o_ctl_b);
    plan_b.withhold = 0;
    int nsm = 152, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = nsm * batch_blocks_per_sm();
    int herr = 0;
    std::vector<int> hvf(n, 0);
    unsigned long long hstats[kStatCount] = {0};
    // graph start; forward kernel start / end; adjoint kernel start / end
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    // inputs: state codes 0..3, finite fields, p_veg / p_den >= -1 (as pf_forward / pf_set_env)
    e = cudaMemsetAsync(arena + o_vf, 0, sizeof(int) * n, st);
    if (e != cudaSuccess) goto cuda_fail;
    for (int k = 0; k < n; ++k) {
        const pf_job& J = jobs[order[k]];
        int* fl = (int*)(arena + o_vf) + k;
        const size_t hw = (size_t)J.H * J.W;
        launch_validate_states(J.S_init, hw, fl, st);
        const float* f[5] = {J.E, J.p_veg, J.p_den, J.V_w, J.theta_w};
        const float lo[5] = {-INFINITY, -1.0f, -1.0f, -INFINITY, -INFINITY};
        for (int i = 0; i < 5; ++i)
            if (f[i]) launch_validate_fields(f[i], hw, lo[i], 1 + i, fl, st);
    }
    e = cudaMemcpyAsync(hvf.data(), arena + o_vf, sizeof(int) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) goto cuda_fail;
    for (int k = 0; k < n; ++k)
        if (hvf[k]) {
            rc = fail(nullptr, PF_EINVAL,
                      "pf_batch_submit: job %d: state codes other than 0..3, NaN/inf fields, or p_veg/p_den < -1",
                      order[k]);
            goto done;
        }
    // tables (pageable host memory: copied before the capture, synchronously)
    e = cudaMemcpy(arena + o_jobs, hj.data(), sizeof(BatchJobDev) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(arena + o_bs, blk_start.data(), sizeof(long long) * (max_blk + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(arena + o_tp, tile_pref.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(arena + o_jb, jobs_in_blk.data(), sizeof(int) * max_blk, cudaMemcpyHostToDevice);
    if (nb) {
        if (e == cudaSuccess) e = cudaMemcpy(arena + o_jobs_b, hjb.data(), sizeof(BatchJobDev) * nb, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(arena + o_bs_b, blk_start_b.data(), sizeof(long long) * (max_blk_b + 1), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(arena + o_tp_b, tile_pref_b.data(), sizeof(long long) * (nb + 1), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(arena + o_jb_b, jobs_in_blk_b.data(), sizeof(int) * max_blk_b, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && batch_adj_configure() != 0) e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) goto cuda_fail;
    // the whole submission (initial states, prep of every fire, the persistent kernel)
    // is captured into one CUDA graph and launched once
    // (captured on a private stream: the caller's may be the legacy default stream,
    // which cannot capture; the graph is then launched on the caller's stream)
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) goto cuda_fail;
    for (auto& x : ev)
        if (e == cudaSuccess) e = cudaEventCreate(&x);
    if (e != cudaSuccess) goto cuda_fail;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) goto cuda_fail;
    cudaEventRecordWithFlags(ev[0], cs, cudaEventRecordExternal);  // timing nodes of the graph
    cudaMemsetAsync(arena + o_ctl, 0, sizeof(unsigned long long) + sizeof(int) * 4, cs);
    cudaMemsetAsync(arena + o_stats, 0, sizeof(unsigned long long) * kStatCount, cs);
    for (int k = 0; k < n; ++k) {
        const pf_job& J = jobs[order[k]];
        const Lay& L = lay[k];
        cudaMemsetAsync(arena + L.st, 0, 2 * L.stbytes, cs);
        cudaMemsetAsync(arena + L.gen, 0, (size_t)L.tx * L.ty * sizeof(int), cs);
        uint8_t* mask = (uint8_t*)(arena + L.mask);
        if (J.form == PF_DISCRETE) {
            cudaMemcpy2DAsync(arena + L.st, L.P, J.S_init, J.W, J.W, J.H, cudaMemcpyDeviceToDevice, cs);
        } else {
            launch_diff_init(J.S_init, J.H, J.W, L.P, (float*)(arena + L.st), mask, cs);
        }
        PrepArgs g{};
        g.H = J.H; g.W = J.W; g.pitch = L.P;
        g.E = J.E; g.pveg = J.p_veg; g.pden = J.p_den; g.V = J.V_w; g.th = J.theta_w;
        g.burnable = J.form == PF_DIFF ? mask : nullptr;
        g.p_h = J.p_h; g.c1 = J.c1; g.c2 = J.c2; g.a = J.a; g.l = J.l;
        prep_derive(g);
        launch_prep(g, (float*)(arena + L.q), cs);
        if (L.adj) {
            const size_t plane = (size_t)J.H * L.P;
            cudaMemcpyAsync(arena + L.tape, arena + L.st, 2 * plane * sizeof(float), cudaMemcpyDeviceToDevice, cs);
            cudaMemsetAsync(arena + L.gq, 0, 8 * plane * sizeof(float), cs);
            cudaMemsetAsync(arena + L.genb, 0, (size_t)L.btx * L.bty * sizeof(int), cs);
        }
    }
    cudaEventRecordWithFlags(ev[1], cs, cudaEventRecordExternal);
    launch_batch(plan, grid, cs);
    cudaEventRecordWithFlags(ev[2], cs, cudaEventRecordExternal);
    if (nb) {
        // terminal adjoint of each job from dL/da_T and its state at T, then the
        // backward work queue, then each job's chain rule of prep and FP64 reduction
        cudaMemsetAsync(arena + o_ctl_b, 0, sizeof(unsigned long long), cs);
        for (int k : ab) {
            const pf_job& J = jobs[order[k]];
            const BatchJobDev& D = hj[k];
            const size_t plane = (size_t)J.H * lay[k].P;
            const int z = D.nblk & 1;
            launch_adjoint_init(J.dL_da, nullptr, D.tape + (size_t)J.T * 2 * plane, J.H, J.W, lay[k].P, D.lam[z],
                                D.sig[z], cs);
        }
        cudaEventRecordWithFlags(ev[3], cs, cudaEventRecordExternal);
        launch_batch_adj(plan_b, nsm * batch_adj_blocks_per_sm(), cs);
        cudaEventRecordWithFlags(ev[4], cs, cudaEventRecordExternal);
        for (int k : ab) {
            const pf_job& J = jobs[order[k]];
            const Lay& L = lay[k];
            PrepArgs g{};
            g.H = J.H; g.W = J.W; g.pitch = L.P;
            g.E = J.E; g.pveg = J.p_veg; g.pden = J.p_den; g.V = J.V_w; g.th = J.theta_w;
            g.burnable = (uint8_t*)(arena + L.mask);
            g.p_h = J.p_h; g.c1 = J.c1; g.c2 = J.c2; g.a = J.a; g.l = J.l;
            prep_derive(g);
            cudaMemsetAsync(J.grad_params, 0, 4 * sizeof(double), cs);
            if (J.grad_pveg) cudaMemsetAsync(J.grad_pveg, 0, (size_t)J.H * J.W * sizeof(float), cs);
            if (J.grad_pden) cudaMemsetAsync(J.grad_pden, 0, (size_t)J.H * J.W * sizeof(float), cs);
            const int npb = prep_adjoint_blocks(J.H, J.W);
            launch_prep_adjoint(g, hj[k].Gq, (double*)(arena + o_part), J.grad_pveg, J.grad_pden, cs);
            launch_reduce_partials((double*)(arena + o_part), npb, J.grad_params, cs);
        }
    }
    e = cudaStreamEndCapture(cs, &graph);
    if (e != cudaSuccess) goto cuda_fail;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) goto cuda_fail;
    e = cudaGraphLaunch(exec, st);
    if (e != cudaSuccess) goto cuda_fail;
    e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hstats, arena + o_stats, sizeof(hstats), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) goto cuda_fail;
    if (herr) rc = fail(nullptr, PF_ETIMEOUT, "pf_batch_submit: a bounded wait for a neighbouring tile ran out");
    {
        pf_batch_stats_t& B = g_batch_stats;
        B.disc_cell_steps += (long long)hstats[kStatDisc];
        B.disc_skipped += (long long)hstats[kStatDiscSkip];
        B.diff_cell_steps += (long long)hstats[kStatDiff];
        B.diff_skipped += (long long)hstats[kStatDiffSkip];
        B.adj_cell_steps += (long long)hstats[kStatAdj];
        B.adj_skipped += (long long)hstats[kStatAdjSkip];
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[1], ev[2]) == cudaSuccess) B.ms_forward += ms;
        if (nb && cudaEventElapsedTime(&ms, ev[3], ev[4]) == cudaSuccess) B.ms_adjoint += ms;
        if (cudaEventElapsedTime(&ms, ev[0], nb ? ev[4] : ev[2]) == cudaSuccess) B.ms_kernels_from_start += ms;
        cudaGetLastError();
        B.waves += 1;
    }
    goto done;
cuda_fail:
    rc = fail(nullptr, PF_ECUDA, "pf_batch_submit: %s", cudaGetErrorString(e));
    cudaGetLastError();
done:
    if (cs) {
        cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(cs, &cst) == cudaSuccess && cst != cudaStreamCaptureStatusNone) {
            cudaGraph_t g2 = nullptr;
            if (cudaStreamEndCapture(cs, &g2) == cudaSuccess && g2) cudaGraphDestroy(g2);
        }
        cudaStreamDestroy(cs);
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamSynchronize(st);
    for (auto& x : ev)
        if (x) cudaEventDestroy(x);
    cudaFree(arena);
    cudaGetLastError();
    (void)ctx;
    return rc;
}

// jobs of at least this many cells run through a context of their own (temporal-blocked
// kernels) instead of the persistent queue; set by pf_batch_set_direct_cells
constexpr long long kBatchDirectCellsDefault = 1ll << 18;
std::atomic<long long> g_batch_direct_cells{kBatchDirectCellsDefault};

// One batch job as a context of its own would run it: the same results as the queue's
// (the discrete draws use the job's fire_id and run; the differentiable forward uses the
// same update), with the blocked kernels and the context's automatic tuning.
static int batch_run_direct(const pf_job& J, int index, cudaStream_t st, std::vector<double>& host_grads) {
    pf_ctx* c = nullptr;
    int rc = pf_create(&c, J.H, J.W, J.form, 1, J.seed, st);
    if (rc) return fail(nullptr, rc, "pf_batch_submit: job %d: %s", index, pf_last_error(nullptr));
    c->fire_id = J.fire_id;
    c->run0 = J.run;
    auto done = [&](int r) {
        if (r) fail(nullptr, r, "pf_batch_submit: job %d: %s", index, c->err.c_str());
        pf_destroy(c);
        return r;
    };
    if ((rc = pf_set_env(c, J.E, J.p_veg, J.p_den, J.V_w, J.theta_w))) return done(rc);
    if ((rc = pf_set_params(c, J.p_h, J.c1, J.c2, J.a, J.p_continue, J.l))) return done(rc);
    if ((rc = pf_forward(c, J.S_init, J.T, J.S_out))) return done(rc);
    if (J.dL_da) {
        double* g = host_grads.data() + 4 * (size_t)index;
        if ((rc = pf_backward(c, J.dL_da, nullptr, g, J.grad_pveg, J.grad_pden))) return done(rc);
        if (cudaMemcpyAsync(J.grad_params, g, 4 * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) {
            cudaGetLastError();
            return done(PF_ECUDA);
        }
    }
    if ((rc = pf_wait(c))) return done(rc);
    return done(PF_OK);
}

int pf_batch_set_direct_cells(long long min_cells) {
    if (min_cells < 0) return fail(nullptr, PF_EINVAL, "pf_batch_set_direct_cells: min_cells must be >= 0");
    g_batch_direct_cells.store(min_cells);
    return PF_OK;
}

int pf_batch_submit(const pf_job* jobs, int n, void* cuda_stream) {
    g_batch_stats = pf_batch_stats_t{};
    pf_ctx* ctx = nullptr;  // context-free: errors go to pf_last_error(NULL)
    if (n < 0 || (n > 0 && !jobs)) return fail(nullptr, PF_EINVAL, "pf_batch_submit: bad job array");
    if (n == 0) return PF_OK;
    const int kB = batch_steps_per_item(), kTR = batch_tile_rows(), kTC = batch_tile_cols();
    for (int i = 0; i < n; ++i) {
        const pf_job& J = jobs[i];
        if (J.H < 1 || J.W < 1 || J.H > 65536 || J.W > 65536 || (uint64_t)J.H * J.W >= (1ull << 32))
            return fail(nullptr, PF_EINVAL, "pf_batch_submit: job %d: bad grid %dx%d", i, J.H, J.W);
        if (J.T < 0 || (J.form != PF_DISCRETE && J.form != PF_DIFF) || !J.S_init || !J.S_out)
            return fail(nullptr, PF_EINVAL, "pf_batch_submit: job %d: bad T, form or NULL state", i);
        const float v[6] = {J.p_h, J.c1, J.c2, J.a, J.p_continue, J.l};
        for (float x : v)
            if (!std::isfinite(x)) return fail(nullptr, PF_EINVAL, "pf_batch_submit: job %d: non-finite parameter", i);
        if (J.p_h < 0 || J.p_continue < 0 || J.p_continue > 1 || !(J.l > 0))
            return fail(nullptr, PF_EINVAL, "pf_batch_submit: job %d: parameter out of range", i);
        if (J.dL_da && (J.form != PF_DIFF || !J.grad_params))
            return fail(nullptr, PF_EINVAL, "pf_batch_submit: job %d: dL_da needs the differentiable form and grad_params", i);
    }
    // large jobs through contexts of their own, the rest through the persistent queue
    const long long direct_cells = g_batch_direct_cells.load();
    std::vector<pf_job> queued;
    std::vector<int> direct;
    for (int i = 0; i < n; ++i) {
        if ((long long)jobs[i].H * jobs[i].W >= direct_cells) direct.push_back(i);
        else queued.push_back(jobs[i]);
    }
    if (!direct.empty()) {
        cudaStream_t st = (cudaStream_t)cuda_stream;
        std::vector<double> host_grads(4 * (size_t)n, 0.0);
        // the direct jobs' contexts allocate from one stream-ordered pool that keeps what
        // they free until the last job ends: a job reuses the memory of those before it
        // instead of allocating and freeing (and synchronising the device) every time
        cudaMemPool_t pool = nullptr;
        {
            int dev = 0;
            cudaMemPoolProps props{};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            if (cudaGetDevice(&dev) == cudaSuccess) {
                props.location.id = dev;
                if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
                    uint64_t keep = ~0ull;
                    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
                } else {
                    pool = nullptr;
                }
            }
            cudaGetLastError();
        }
        g_ctx_pool = pool;
        cudaEvent_t d0 = nullptr, d1 = nullptr;
        const bool timing = cudaEventCreate(&d0) == cudaSuccess && cudaEventCreate(&d1) == cudaSuccess;
        if (timing) cudaEventRecord(d0, st);
        int rc = PF_OK;
        for (int i : direct) {
            if ((rc = batch_run_direct(jobs[i], i, st, host_grads))) break;
            pf_batch_stats_t& B = g_batch_stats;
            const long long cs = (long long)jobs[i].H * jobs[i].W * jobs[i].T;
            B.direct_jobs += 1;
            B.direct_cell_steps += cs * (jobs[i].dL_da ? 2 : 1);
        }
        if (timing) {
            cudaEventRecord(d1, st);
            float ms = 0.f;
            if (cudaEventSynchronize(d1) == cudaSuccess && cudaEventElapsedTime(&ms, d0, d1) == cudaSuccess)
                g_batch_stats.ms_direct += ms;
        }
        if (d0) cudaEventDestroy(d0);
        if (d1) cudaEventDestroy(d1);
        cudaGetLastError();
        g_ctx_pool = nullptr;
        if (cudaStreamSynchronize(st) != cudaSuccess && rc == PF_OK)
            rc = fail(nullptr, PF_ECUDA, "pf_batch_submit: %s", cudaGetErrorString(cudaGetLastError()));
        if (pool) cudaMemPoolDestroy(pool);  // every context freed its memory into it
        cudaGetLastError();
        if (rc) return rc;
        if (queued.empty()) return PF_OK;
        jobs = queued.data();
        n = (int)queued.size();
    }
    // Device memory of one job in a wave's arena (as batch_submit_wave lays it out): two
    // state buffers, q, the burnable mask, tile counters and, with an adjoint, every
    // state, the scaled adjoint and dL/dq.
    auto job_bytes = [&](const pf_job& J) {
        const size_t P = (size_t)pitch_of(J.W), plane = (size_t)J.H * P;
        auto r = [](size_t b) { return (b + 255) & ~(size_t)255; };
        const size_t tiles = (size_t)((J.W + kTC - 1) / kTC) * ((J.H + kTR - 1) / kTR);
        size_t b = r(2 * (J.form == PF_DISCRETE ? plane : 2 * plane * sizeof(float))) + r(8 * plane * sizeof(float)) +
                   r((size_t)J.H * J.W) + r(tiles * sizeof(int));
        if (J.dL_da) {
            const size_t bt = (size_t)((J.W + batch_adj_tile_cols() - 1) / batch_adj_tile_cols()) *
                              ((J.H + batch_adj_tile_rows() - 1) / batch_adj_tile_rows());
            b += r((size_t)(J.T + 1) * 2 * plane * sizeof(float)) + r(2 * 2 * plane * sizeof(float)) + r(2 * plane) +
                 r(8 * plane * sizeof(float)) + r(bt * sizeof(int));
        }
        return b + 4096;  // and its share of the plan tables
    };
    // Jobs whose arenas do not fit in the device memory together run in waves, each a
    // submission of its own; a wave takes the largest remaining jobs that fit in 70% of
    // the free memory.
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        free_b = 0;
    }
    const size_t budget = (size_t)(0.7 * (double)free_b);
    std::vector<int> by_size(n);
    for (int i = 0; i < n; ++i) by_size[i] = i;
    std::stable_sort(by_size.begin(), by_size.end(),
                     [&](int x, int y) { return job_bytes(jobs[x]) > job_bytes(jobs[y]); });
    std::vector<char> done(n, 0);
    int left = n;
    std::vector<pf_job> wave;
    while (left > 0) {
        wave.clear();
        size_t used = 0;
        for (int i : by_size) {
            if (done[i]) continue;
            const size_t b = job_bytes(jobs[i]);
            if (wave.empty() || used + b <= budget) {
                wave.push_back(jobs[i]);
                used += b;
                done[i] = 1;
                --left;
            }
        }
        const int rc = batch_submit_wave(wave.data(), (int)wave.size(), (cudaStream_t)cuda_stream);
        if (rc) return rc;
    }
    return PF_OK;
}

int pf_batch_last_stats(pf_batch_stats_t* out) {
    if (!out) return fail(nullptr, PF_EINVAL, "pf_batch_last_stats: out is NULL");
    *out = g_batch_stats;
    return PF_OK;
}

}  // extern "C"
