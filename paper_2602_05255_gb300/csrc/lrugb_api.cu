// C-ABI of the library (include/lrugb.h): argument validation, state
// allocation, and the launch sequence of each call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lrugb.h"
#include "common.cuh"
#include "internal.h"

using namespace lru;

namespace {
// An NVTX range around each C-ABI call (named after the call), so that a
// profiler's timeline groups the kernels of a call under it.  NVTX is
// header-only and costs nothing when no profiler is attached.
struct NvtxScope {
    explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
};
}  // namespace
#define LRU_RANGE() NvtxScope lru_nvtx_scope_(__func__)

namespace {

constexpr int MAXKK = 16;
constexpr int MAXN = 2048;
constexpr int MAXKC = 64;
constexpr size_t CANARY_BYTES = 256;   // debug build: guard zone after each region of a handle's allocation

size_t dtype_size(int d) {
    switch (d) {
        case LRU_F64: return 8;
        case LRU_C128: return 16;
        case LRU_F32: return 4;
        case LRU_C64: return 8;
        default: return 0;
    }
}

size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

}  // namespace

struct lru_ctx {
    lru_config cfg;
    int dtype = 0;
    bool pf = false, delayed = false;
    int W = 0, kk = 0, K = 0, Kc = 0, Kc32 = 0, flush = 0;
    bool split_bf16 = false;
    bool df = false;             // double-float GEMV (F64 handles)
    int device = 0;
    cudaStream_t stream = nullptr;
    int n_uni = 0, n_max = 0;
    std::vector<int> n_h, kv_h;
    std::vector<long long> moff_h, voff_h;
    long long sum_n = 0, sum_n2 = 0;
    // device memory
    unsigned char* base = nullptr;
    size_t bytes = 0, persist_bytes = 0;
    int* d_n = nullptr;
    long long* d_moff = nullptr;
    long long* d_voff = nullptr;
    int* d_kv = nullptr;
    int* d_items = nullptr;
    int nitems = 0;
    // persistent step: propose order, accept items (largest walkers first), control block
    int* d_order = nullptr;
    int* d_sitems = nullptr;
    int* d_nacc_w = nullptr;
    int* d_ctl = nullptr;        // counter, prop_done[W], items_done[W], fin[W], flush_done[W]
    int* d_fitems = nullptr;     // delayed: flush strips (walker, 32-column block)
    int* d_nflush_w = nullptr;
    int nflush = 0;
    uint8_t* d_acc = nullptr;
    int* d_never = nullptr;      // a flag no kernel writes (bounded-wait self-test)
    bool items_smem = true;
    void *G = nullptr, *P = nullptr, *Q = nullptr;
    float *P32h = nullptr, *P32l = nullptr, *Q32h = nullptr, *Q32l = nullptr;
    int* tau = nullptr;
    double* logabs = nullptr;
    void* sgn = nullptr;
    void *X = nullptr, *Rinv = nullptr, *ratio = nullptr, *VP = nullptr, *QtU = nullptr;
    int* pst = nullptr;
    int* err = nullptr;
    // refresh workspace (allocated on first use)
    void* ws = nullptr;
    int nws = 0;
    // profiling: event pairs per kernel class, and a launch counter
    bool prof_on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev[LRU_PROF_CLASSES];
    size_t prof_used[LRU_PROF_CLASSES] = {};
    long long launches = 0;
    // last proposal
    bool has_prop = false;
    DevOperand lastV{};
    const void* lastC = nullptr;
    // workspace of the tensor-core refresh (allocated on first use)
    void* ozw = nullptr;
    size_t oz_bytes = 0;
    void* ozM = nullptr;         // fresh inverses when the drift is asked for
    size_t ozM_bytes = 0;
    bool oz_ok = false;          // the tensor-core refresh applies to this handle
    // adjoint workspace (allocated on first use)
    void* bws = nullptr;
    int n_sm = 148;
    // debug build: offsets of the guard zones between the regions of the allocation
    std::vector<size_t> canaries;

    DevLayout layout() const {
        DevLayout L;
        L.W = W;
        L.n_uni = n_uni;
        L.n_max = n_max;
        L.n = d_n;
        L.moff = d_moff;
        L.voff = d_voff;
        L.kk = kk;
        L.kvec = d_kv;
        L.Kc = Kc;
        L.K = K;
        L.Kc32 = Kc32;
        L.rows = sum_n;
        return L;
    }
    template <typename T>
    DevState<T> state() const {
        DevState<T> S;
        S.G = (T*)G;
        S.P = (T*)P;
        S.Q = (T*)Q;
        S.split_bf16 = split_bf16 ? 1 : 0;
        S.P32h = P32h;
        S.P32l = P32l;
        S.Q32h = Q32h;
        S.Q32l = Q32l;
        S.tau = tau;
        S.logabs = logabs;
        S.sgn = (T*)sgn;
        S.X = (T*)X;
        S.Rinv = (T*)Rinv;
        S.ratio = (T*)ratio;
        S.pst = pst;
        S.VP = (T*)VP;
        S.QtU = (T*)QtU;
        S.err = err;
        return S;
    }
};

#define LRU_DISPATCH(ctx, ...)                      \
    switch ((ctx)->dtype) {                         \
        case LRU_F64: { using T = double; __VA_ARGS__; } break;   \
        case LRU_C128: { using T = lru::c128; __VA_ARGS__; } break; \
        case LRU_F32: { using T = float; __VA_ARGS__; } break;    \
        case LRU_C64: { using T = lru::c64; __VA_ARGS__; } break; \
        default: return LRU_ERR_ARG;                \
    }

static lru_status cuda_check() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LRU_OK : LRU_ERR_CUDA;
}

#define CK(call)                                                     \
    do {                                                             \
        if ((call) != cudaSuccess) { cudaGetLastError(); return LRU_ERR_CUDA; } \
    } while (0)

static void prof_begin(lru_ctx* h, int cls) {
    if (!h->prof_on) return;
    auto& v = h->prof_ev[cls];
    if (h->prof_used[cls] == v.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) { cudaGetLastError(); return; }
        v.emplace_back(a, b);
    }
    cudaEventRecord(v[h->prof_used[cls]].first, h->stream);
}

static void prof_end(lru_ctx* h, int cls) {
    if (!h->prof_on) return;
    auto& v = h->prof_ev[cls];
    if (h->prof_used[cls] < v.size()) cudaEventRecord(v[h->prof_used[cls]++].second, h->stream);
}

static lru_status ensure_ws(lru_ctx* h) {
    if (h->ws) return LRU_OK;
    int nws = std::min(h->W, 2 * h->n_sm);
    size_t b = (size_t)nws * h->n_max * h->n_max * dtype_size(h->dtype);
    if (cudaMalloc(&h->ws, b) != cudaSuccess) {
        cudaGetLastError();
        h->ws = nullptr;
        return LRU_ERR_NOMEM;
    }
    h->nws = nws;
    return LRU_OK;
}

extern "C" {

const char* lru_status_string(lru_status s) {
    switch (s) {
        case LRU_OK: return "ok";
        case LRU_ERR_ARG: return "invalid argument";
        case LRU_ERR_CUDA: return "CUDA runtime error";
        case LRU_ERR_NOMEM: return "device allocation failed";
        case LRU_ERR_STATE: return "call out of order";
        case LRU_ERR_SINGULAR: return "singular matrix";
        case LRU_ERR_NOT_SKEW: return "matrix is not skew-symmetric";
        case LRU_ERR_TIMEOUT: return "bounded device wait gave up";
        case LRU_ERR_UNSUPPORTED: return "combination not supported";
    }
    return "unknown status";
}

#ifdef LRU_DEBUG
const char* lru_version(void) { return "lrugb 0.2.0 sm_103a debug"; }
#else
const char* lru_version(void) { return "lrugb 0.2.0 sm_103a"; }
#endif

lru_status lru_create(const lru_config* cfg, lru_handle* out) {
    LRU_RANGE();
    if (!cfg || !out) return LRU_ERR_ARG;
    *out = nullptr;
    if (cfg->kind != LRU_DET && cfg->kind != LRU_PF) return LRU_ERR_ARG;
    if (dtype_size(cfg->dtype) == 0) return LRU_ERR_ARG;
    if (cfg->walkers < 1 || cfg->walkers > (1 << 24)) return LRU_ERR_ARG;
    if (cfg->k < 1) return LRU_ERR_ARG;
    const int kk = cfg->kind == LRU_PF ? 2 * cfg->k : cfg->k;
    if (kk > MAXKK) return LRU_ERR_ARG;
    if (cfg->delay < 0) return LRU_ERR_ARG;
    if (cfg->flush < LRU_FLUSH_NATIVE || cfg->flush > LRU_FLUSH_SPLIT) return LRU_ERR_ARG;
    if (cfg->arith != LRU_ARITH_NATIVE && cfg->arith != LRU_ARITH_DF) return LRU_ERR_ARG;
    if (cfg->tile_chunks < 0) return LRU_ERR_ARG;
    if (cfg->refresh < LRU_REFRESH_AUTO || cfg->refresh > LRU_REFRESH_TENSOR) return LRU_ERR_ARG;
    const bool delayed = cfg->delay >= 2;
    if (delayed && cfg->delay * kk > MAXKC) return LRU_ERR_ARG;
    if (cfg->flush != LRU_FLUSH_NATIVE && !(delayed && cfg->dtype == LRU_F64)) return LRU_ERR_UNSUPPORTED;
    if (cfg->flush == LRU_FLUSH_DF && !(delayed && cfg->dtype == LRU_F64)) return LRU_ERR_UNSUPPORTED;

    lru_ctx* h = new (std::nothrow) lru_ctx();
    if (!h) return LRU_ERR_NOMEM;
    h->cfg = *cfg;
    h->cfg.n_per_walker = nullptr;
    h->cfg.k_per_walker = nullptr;
    h->dtype = cfg->dtype;
    h->pf = cfg->kind == LRU_PF;
    h->delayed = delayed;
    h->W = (int)cfg->walkers;
    h->kk = kk;
    h->K = delayed ? cfg->delay : 0;
    h->Kc = delayed ? cfg->delay * kk : 0;
    const bool bf16 = cfg->flush == LRU_FLUSH_BF16 || cfg->flush == LRU_FLUSH_BF16X3;
    h->split_bf16 = bf16;
    h->Kc32 = bf16 ? (h->Kc + 63) / 64 * 64 : (h->Kc + 31) / 32 * 32;
    h->flush = cfg->flush;
    h->device = cfg->device;
    h->df = cfg->arith == LRU_ARITH_DF && cfg->dtype == LRU_F64;

    // geometry
    h->n_h.resize(h->W);
    h->kv_h.resize(h->W);
    for (int w = 0; w < h->W; ++w) {
        int n = cfg->n_per_walker ? cfg->n_per_walker[w] : cfg->n;
        int kw = cfg->k_per_walker ? cfg->k_per_walker[w] : cfg->k;
        if (n < 1 || n > MAXN || kw < 1 || kw > cfg->k || (h->pf && (n & 1))) {
            delete h;
            return LRU_ERR_ARG;
        }
        h->n_h[w] = n;
        h->kv_h[w] = h->pf ? 2 * kw : kw;
    }
    bool uniform = true;
    for (int w = 1; w < h->W; ++w) uniform = uniform && h->n_h[w] == h->n_h[0];
    h->n_uni = uniform ? h->n_h[0] : 0;
    h->n_max = *std::max_element(h->n_h.begin(), h->n_h.end());
    h->moff_h.resize(h->W);
    h->voff_h.resize(h->W);
    for (int w = 0; w < h->W; ++w) {
        h->moff_h[w] = h->sum_n2;
        h->voff_h[w] = h->sum_n;
        h->sum_n2 += (long long)h->n_h[w] * h->n_h[w];
        h->sum_n += h->n_h[w];
    }
    bool kuni = true;
    for (int w = 0; w < h->W; ++w) kuni = kuni && h->kv_h[w] == kk;
    if (!uniform && h->pf) { /* ragged Pfaffian handles are allowed */ }
    {
        const int n = h->n_uni;
        // the split-product kernels: F64, uniform n % 128 == 0 up to 2048
        const bool shape = h->dtype == LRU_F64 && n > 0 && n % 128 == 0 && n >= 128 && n <= 2048 && h->W <= 65535;
        const bool fits = shape && !h->pf;   // the tensor-core refresh: determinants
        if (cfg->refresh == LRU_REFRESH_TENSOR && !fits) { delete h; return LRU_ERR_UNSUPPORTED; }
        h->oz_ok = fits && cfg->refresh != LRU_REFRESH_FP64;
        if (cfg->flush == LRU_FLUSH_SPLIT && !(shape && delayed && h->Kc <= 64)) { delete h; return LRU_ERR_UNSUPPORTED; }
    }

    if (cudaSetDevice(h->device) != cudaSuccess) { cudaGetLastError(); delete h; return LRU_ERR_CUDA; }
    {
        int nsm = 0;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device) == cudaSuccess && nsm > 0)
            h->n_sm = nsm;
        cudaGetLastError();
    }

    // accept work items: (walker, first chunk, end chunk, use_smem)
    std::vector<int> items;
    const size_t sz = dtype_size(h->dtype);
    h->items_smem = (size_t)2 * kk * h->n_max * sz <= 160 * 1024;
    for (int w = 0; w < h->W; ++w) {
        const int n = h->n_h[w];
        const int ch = cfg->tile_chunks > 0 ? std::min(cfg->tile_chunks, 256)
                                            : std::max(8, std::min(64, n / 4));
        for (int l0 = 0; l0 < n; l0 += ch) {
            items.push_back(w);
            items.push_back(l0);
            items.push_back(std::min(n, l0 + ch));
            items.push_back(h->items_smem ? 1 : 0);
        }
    }
    h->nitems = (int)items.size() / 4;
    // persistent-step queue: walkers by decreasing n^2 k (longest first)
    std::vector<int> order(h->W), nacc_w(h->W, 0), sitems;
    for (int w = 0; w < h->W; ++w) order[w] = w;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (long long)h->n_h[a] * h->n_h[a] * h->kv_h[a] > (long long)h->n_h[b] * h->n_h[b] * h->kv_h[b];
    });
    for (size_t q = 0; q < items.size(); q += 4) nacc_w[items[q]] += 1;
    {
        std::vector<std::vector<int>> per(h->W);
        for (size_t q = 0; q < items.size(); q += 4)
            for (int c = 0; c < 4; ++c) per[items[q]].push_back(items[q + c]);
        for (int w : order) sitems.insert(sitems.end(), per[w].begin(), per[w].end());
    }
    // delayed form: flush strips of 32 columns of A_0^{-1}, largest walkers first
    std::vector<int> fitems, nflush_w(h->W, 0);
    if (delayed)
        for (int w : order) {
            const int nt = (h->n_h[w] + 31) / 32;
            for (int t = nt - 1; t >= 0; --t) {
                fitems.push_back(w);
                fitems.push_back(t);
            }
            nflush_w[w] = nt;
        }
    h->nflush = (int)fitems.size() / 2;

    // one allocation: persistent state first, then scratch and metadata
    const bool tc = delayed && cfg->flush != LRU_FLUSH_NATIVE && cfg->flush != LRU_FLUSH_DF &&
                    cfg->flush != LRU_FLUSH_SPLIT;
    size_t off = 0;
#ifdef LRU_DEBUG
    // every region is followed by a guard zone of CANARY_BYTES bytes of 0xA5
    // that lru_check_device_error verifies
    auto take = [&](size_t b) {
        size_t o = off;
        off = align_up(off + b);
        h->canaries.push_back(off);
        off = align_up(off + CANARY_BYTES);
        return o;
    };
#else
    auto take = [&](size_t b) { size_t o = off; off = align_up(off + b); return o; };
#endif
    const size_t oG = take((size_t)h->sum_n2 * sz);
    const size_t oP = delayed ? take((size_t)h->sum_n * h->Kc * sz) : 0;
    const size_t oQ = delayed ? take((size_t)h->sum_n * h->Kc * sz) : 0;
    const size_t o32 = tc ? take((size_t)4 * h->sum_n * h->Kc32 * (h->split_bf16 ? 2 : sizeof(float))) : 0;
    const size_t oTau = take((size_t)h->W * sizeof(int));
    const size_t oLog = take((size_t)h->W * sizeof(double));
    const size_t oSgn = take((size_t)h->W * sz);
    h->persist_bytes = off;
    const size_t oX = take((size_t)h->sum_n * kk * sz);
    const size_t oRinv = take((size_t)h->W * MAXKK * MAXKK * sz);
    const size_t oRatio = take((size_t)h->W * sz);
    const size_t oPst = take((size_t)h->W * sizeof(int));
    const size_t oVP = delayed ? take((size_t)h->W * MAXKK * h->Kc * sz) : 0;
    const size_t oQtU = delayed ? take((size_t)h->W * h->Kc * MAXKK * sz) : 0;
    const size_t oErr = take(sizeof(int));
    const size_t oN = take((size_t)h->W * sizeof(int));
    const size_t oMoff = take((size_t)h->W * sizeof(long long));
    const size_t oVoff = take((size_t)h->W * sizeof(long long));
    const size_t oKv = take((size_t)h->W * sizeof(int));
    const size_t oItems = take(items.size() * sizeof(int));
    const size_t oOrder = take((size_t)h->W * sizeof(int));
    const size_t oSItems = take(sitems.size() * sizeof(int));
    const size_t oNacc = take((size_t)h->W * sizeof(int));
    const size_t oCtl = take((size_t)(1 + 4 * h->W) * sizeof(int));
    const size_t oFit = take(std::max<size_t>(fitems.size(), 2) * sizeof(int));
    const size_t oNfl = take((size_t)h->W * sizeof(int));
    const size_t oAcc = take((size_t)h->W);
    const size_t oNever = take(sizeof(int));
    h->bytes = off;
    if (cudaMalloc(&h->base, h->bytes) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return LRU_ERR_NOMEM;
    }
    unsigned char* b = h->base;
    h->G = b + oG;
    if (delayed) { h->P = b + oP; h->Q = b + oQ; }
    if (tc) {
        const size_t e = (size_t)h->sum_n * h->Kc32 * (h->split_bf16 ? 2 : sizeof(float));   // bytes
        h->P32h = (float*)(b + o32);
        h->P32l = (float*)(b + o32 + e);
        h->Q32h = (float*)(b + o32 + 2 * e);
        h->Q32l = (float*)(b + o32 + 3 * e);
    }
    h->tau = (int*)(b + oTau);
    h->logabs = (double*)(b + oLog);
    h->sgn = b + oSgn;
    h->X = b + oX;
    h->Rinv = b + oRinv;
    h->ratio = b + oRatio;
    h->pst = (int*)(b + oPst);
    if (delayed) { h->VP = b + oVP; h->QtU = b + oQtU; }
    h->err = (int*)(b + oErr);
    h->d_n = (int*)(b + oN);
    h->d_moff = (long long*)(b + oMoff);
    h->d_voff = (long long*)(b + oVoff);
    h->d_kv = kuni ? nullptr : (int*)(b + oKv);
    h->d_items = (int*)(b + oItems);
    h->d_order = (int*)(b + oOrder);
    h->d_sitems = (int*)(b + oSItems);
    h->d_nacc_w = (int*)(b + oNacc);
    h->d_ctl = (int*)(b + oCtl);
    h->d_fitems = (int*)(b + oFit);
    h->d_nflush_w = (int*)(b + oNfl);
    h->d_acc = (uint8_t*)(b + oAcc);
    h->d_never = (int*)(b + oNever);
    lru_status s = LRU_OK;
    if (cudaMemset(h->base, 0, h->bytes) != cudaSuccess ||
        cudaMemcpy(h->d_n, h->n_h.data(), h->W * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_moff, h->moff_h.data(), h->W * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_voff, h->voff_h.data(), h->W * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b + oKv, h->kv_h.data(), h->W * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_items, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_order, order.data(), h->W * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_sitems, sitems.data(), sitems.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_nacc_w, nacc_w.data(), h->W * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        (!fitems.empty() &&
         cudaMemcpy(h->d_fitems, fitems.data(), fitems.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaMemcpy(h->d_nflush_w, nflush_w.data(), h->W * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
        s = LRU_ERR_CUDA;
#ifdef LRU_DEBUG
    for (size_t c : h->canaries)
        if (s == LRU_OK && cudaMemset(h->base + c, 0xA5, CANARY_BYTES) != cudaSuccess) s = LRU_ERR_CUDA;
#endif
    if (s != LRU_OK) {
        cudaGetLastError();
        cudaFree(h->base);
        delete h;
        return s;
    }
    *out = h;
    return LRU_OK;
}

lru_status lru_destroy(lru_handle h) {
    LRU_RANGE();
    if (!h) return LRU_ERR_ARG;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    cudaFree(h->base);
    if (h->ws) cudaFree(h->ws);
    if (h->bws) cudaFree(h->bws);
    if (h->ozw) cudaFree(h->ozw);
    if (h->ozM) cudaFree(h->ozM);
    for (auto& v : h->prof_ev)
        for (auto& e : v) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    cudaGetLastError();
    delete h;
    return LRU_OK;
}

lru_status lru_set_stream(lru_handle h, void* stream) {
    LRU_RANGE();
    if (!h) return LRU_ERR_ARG;
    h->stream = (cudaStream_t)stream;
    return LRU_OK;
}

lru_status lru_device_bytes(lru_handle h, size_t* bytes) {
    LRU_RANGE();
    if (!h || !bytes) return LRU_ERR_ARG;
    *bytes = h->bytes + (h->ws ? (size_t)h->nws * h->n_max * h->n_max * dtype_size(h->dtype) : 0) + h->oz_bytes + h->ozM_bytes;
    return LRU_OK;
}

static void oz_prof_hook(void* p, int cls, int begin) {
    lru_ctx* h = (lru_ctx*)p;
    if (begin) prof_begin(h, cls);
    else prof_end(h, cls);
}

static lru_status ensure_oz(lru_ctx* h) {
    if (h->ozw) return LRU_OK;
    const size_t b = oz_work_bytes(h->W, h->n_uni);
    if (cudaMalloc(&h->ozw, b) != cudaSuccess) {
        cudaGetLastError();
        h->ozw = nullptr;
        return LRU_ERR_NOMEM;
    }
    h->oz_bytes = b;
    return LRU_OK;
}

static lru_status do_init(lru_handle h, const void* A, const uint8_t* mask, double* drift, double* logabs_out,
                          void* sign_out, bool with_ws) {
    if (!A) return LRU_ERR_ARG;
    CK(cudaSetDevice(h->device));
    if (h->oz_ok) {
        // FP64 panels + tensor-core trailing updates: in place in the state, or
        // (drift asked for) into a workspace compared with the tracked inverse
        lru_status s = ensure_oz(h);
        if (s != LRU_OK) return s;
        if (drift && !h->ozM) {
            const size_t b = (size_t)h->W * h->n_uni * h->n_uni * sizeof(double);
            if (cudaMalloc(&h->ozM, b) != cudaSuccess) {
                cudaGetLastError();
                h->ozM = nullptr;
                return LRU_ERR_NOMEM;
            }
            h->ozM_bytes = b;
        }
        OzWork Z{};
        oz_work_carve(Z, h->ozw, h->W, h->n_uni);
        Z.M = drift ? (double*)h->ozM : (double*)h->G;
        DevState<double> S = h->state<double>();
        prof_begin(h, LRU_PROF_REFRESH);
        bool ok = launch_refresh_oz(h->W, h->n_uni, (const double*)A, Z, S, mask, h->delayed, !drift, h->err,
                                    h->stream, h->prof_on ? oz_prof_hook : nullptr, h);
        if (ok && drift)
            launch_oz_drift_store(h->W, h->n_uni, h->layout(), S, Z.M, mask, drift, h->delayed, h->stream);
        prof_end(h, LRU_PROF_REFRESH);
        if (ok) {
            h->launches += 2 + 4 * (h->n_uni / OZ_B);
            s = cuda_check();
            if (s != LRU_OK) return s;
            if (logabs_out)
                CK(cudaMemcpyAsync(logabs_out, h->logabs, h->W * sizeof(double), cudaMemcpyDefault, h->stream));
            if (sign_out) CK(cudaMemcpyAsync(sign_out, h->sgn, h->W * sizeof(double), cudaMemcpyDefault, h->stream));
            h->has_prop = false;
            return LRU_OK;
        }
        cudaGetLastError();   // tensor maps unavailable: the FP64 form below
    }
    if (with_ws || h->pf) {
        lru_status s = ensure_ws(h);
        if (s != LRU_OK) return s;
    }
    DevLayout L = h->layout();
    prof_begin(h, LRU_PROF_REFRESH);
    h->launches += h->pf ? 2 : 1;
    LRU_DISPATCH(h, {
        DevState<T> S = h->state<T>();
        launch_refresh<T>(h->pf, h->delayed, L, S, (const T*)A, mask, with_ws ? (T*)h->ws : nullptr, h->nws,
                          drift, !h->pf, h->stream);
        if (h->pf) launch_slogpf<T>(L, (const T*)A, mask, (T*)h->ws, h->nws, S.logabs, S.sgn, h->stream);
    });
    prof_end(h, LRU_PROF_REFRESH);
    lru_status s = cuda_check();
    if (s != LRU_OK) return s;
    const size_t sz = dtype_size(h->dtype);
    if (logabs_out) CK(cudaMemcpyAsync(logabs_out, h->logabs, h->W * sizeof(double), cudaMemcpyDefault, h->stream));
    if (sign_out) CK(cudaMemcpyAsync(sign_out, h->sgn, h->W * sz, cudaMemcpyDefault, h->stream));
    h->has_prop = false;
    return LRU_OK;
}

lru_status lru_init_det(lru_handle h, const void* A, double* logabs, void* sign) {
    LRU_RANGE();
    if (!h) return LRU_ERR_ARG;
    if (h->pf) return LRU_ERR_STATE;
    return do_init(h, A, nullptr, nullptr, logabs, sign, false);
}

lru_status lru_init_pf(lru_handle h, const void* A, double* logabs, void* sign) {
    LRU_RANGE();
    if (!h) return LRU_ERR_ARG;
    if (!h->pf) return LRU_ERR_STATE;
    return do_init(h, A, nullptr, nullptr, logabs, sign, false);
}

lru_status lru_refresh_from_scratch(lru_handle h, const void* A, const uint8_t* mask, double* drift) {
    LRU_RANGE();
    if (!h) return LRU_ERR_ARG;
    return do_init(h, A, mask, drift, nullptr, nullptr, true);
}

// 1 if exactly one slot of the operand is dense (launch_propose then runs that
// column's pass over A^{-1} as its own kernel), else 0
static int one_dense_column(unsigned onehot_mask, int kk) {
    const unsigned all = (kk >= 32) ? 0xffffffffu : ((1u << kk) - 1u);
    const unsigned dense = ~onehot_mask & all;
    return (dense != 0 && (dense & (dense - 1)) == 0) ? 1 : 0;
}

static bool operand_ok(const lru_operand* o, int kk) {
    if (!o) return false;
    const unsigned all = (kk >= 32) ? 0xffffffffu : ((1u << kk) - 1u);
    const unsigned m = o->onehot_mask & all;
    if (m != 0 && !o->idx) return false;
    if (m != all && !o->dense) return false;
    return true;
}

lru_status lru_propose_det(lru_handle h, const lru_operand* U, const lru_operand* V, void* ratio, int32_t* st) {
    LRU_RANGE();
    if (!h || !ratio) return LRU_ERR_ARG;
    if (h->pf) return LRU_ERR_STATE;
    if (!operand_ok(U, h->kk) || !operand_ok(V, h->kk)) return LRU_ERR_ARG;
    CK(cudaSetDevice(h->device));
    DevOperand dU{U->dense, U->idx, U->onehot_mask, h->kk};
    DevOperand dV{V->dense, V->idx, V->onehot_mask, h->kk};
    DevLayout L = h->layout();
    const unsigned all = (1u << h->kk) - 1u;
    h->launches += 1 + ((h->delayed && (dU.mask & all) != all) ? 1 : 0) + one_dense_column(dU.mask, h->kk);
    prof_begin(h, LRU_PROF_PROPOSE);
    LRU_DISPATCH(h, {
        launch_propose<T>(false, h->delayed, h->df, L, h->state<T>(), dU, dV, nullptr, (T*)ratio, st, h->stream);
    });
    prof_end(h, LRU_PROF_PROPOSE);
    lru_status s = cuda_check();
    if (s != LRU_OK) return s;
    h->lastV = dV;
    h->has_prop = true;
    return LRU_OK;
}

lru_status lru_propose_pf(lru_handle h, const lru_operand* B, const void* C, void* ratio, int32_t* st) {
    LRU_RANGE();
    if (!h || !ratio) return LRU_ERR_ARG;
    if (!h->pf) return LRU_ERR_STATE;
    if (!operand_ok(B, h->kk)) return LRU_ERR_ARG;
    CK(cudaSetDevice(h->device));
    DevOperand dB{B->dense, B->idx, B->onehot_mask, h->kk};
    DevLayout L = h->layout();
    const unsigned all = (1u << h->kk) - 1u;
    h->launches += 1 + ((h->delayed && (dB.mask & all) != all) ? 1 : 0) + one_dense_column(dB.mask, h->kk);
    prof_begin(h, LRU_PROF_PROPOSE);
    LRU_DISPATCH(h, {
        launch_propose<T>(true, h->delayed, h->df, L, h->state<T>(), dB, dB, (const T*)C, (T*)ratio, st, h->stream);
    });
    prof_end(h, LRU_PROF_PROPOSE);
    lru_status s = cuda_check();
    if (s != LRU_OK) return s;
    h->lastV = dB;
    h->lastC = C;
    h->has_prop = true;
    return LRU_OK;
}

lru_status lru_step_persistent(lru_handle h, const lru_operand* U, const lru_operand* V, const void* C,
                               int32_t accept, const uint8_t* mask, const double* u, void* ratio, int32_t* st,
                               uint8_t* acc_out) {
    LRU_RANGE();
    if (!h || !ratio) return LRU_ERR_ARG;
    if (!operand_ok(U, h->kk)) return LRU_ERR_ARG;
    if (!h->pf && !operand_ok(V, h->kk)) return LRU_ERR_ARG;
    CK(cudaSetDevice(h->device));
    DevOperand dU{U->dense, U->idx, U->onehot_mask, h->kk};
    DevOperand dV = h->pf ? dU : DevOperand{V->dense, V->idx, V->onehot_mask, h->kk};
    StepCtl ctl;
    ctl.counter = h->d_ctl;
    ctl.prop_done = h->d_ctl + 1;
    ctl.items_done = h->d_ctl + 1 + h->W;
    ctl.fin = h->d_ctl + 1 + 2 * h->W;
    ctl.flush_done = h->d_ctl + 1 + 3 * h->W;
    ctl.acc = acc_out ? acc_out : h->d_acc;
    ctl.order = h->d_order;
    ctl.acc_items = reinterpret_cast<const int4*>(h->d_sitems);
    ctl.nacc_w = h->d_nacc_w;
    ctl.nacc = h->nitems;
    ctl.flush_items = reinterpret_cast<const int2*>(h->d_fitems);
    ctl.nflush_w = h->d_nflush_w;
    ctl.nflush = h->nflush;
    ctl.do_accept = accept != 0;
    ctl.mask = mask;
    ctl.u = u;
    CK(cudaMemsetAsync(h->d_ctl, 0, (size_t)(1 + 4 * h->W) * sizeof(int), h->stream));
    DevLayout L = h->layout();
    h->launches += 1;
    prof_begin(h, LRU_PROF_PROPOSE);
    LRU_DISPATCH(h, {
        launch_step<T>(h->pf, h->delayed, L, h->state<T>(), dU, dV, (const T*)C, (T*)ratio, st, ctl, 2 * h->n_sm,
                       h->stream);
    });
    prof_end(h, LRU_PROF_PROPOSE);
    lru_status s = cuda_check();
    if (s != LRU_OK) return s;
    h->lastV = dV;
    h->lastC = C;
    h->has_prop = true;
    return LRU_OK;
}

static lru_status do_flush(lru_handle h, const uint8_t* force) {
    DevLayout L = h->layout();
    prof_begin(h, LRU_PROF_FLUSH);
    h->launches += 2;
    if (h->flush == LRU_FLUSH_SPLIT) {
        lru_status s = ensure_oz(h);
        if (s != LRU_OK) { prof_end(h, LRU_PROF_FLUSH); return s; }
        OzWork Z{};
        oz_work_carve(Z, h->ozw, h->W, h->n_uni);
        Z.M = (double*)h->G;
        h->launches += 4;   // flush flags, column balance, two slicings, GEMM (+ finish counted above)
        // determinant: A_0^{-1} -= P Q^T (Eq. delayed_Ainv); Pfaffian: A_0^{-1} += P Q^T
        // (Eq. pf_delayed_Ainv), then the lower triangle mirrored from the upper
        if (!launch_flush_split(h->W, h->n_uni, h->K, h->Kc, h->kk, (const double*)h->P, (const double*)h->Q,
                                h->pf ? 1.0 : -1.0, h->tau, force, Z, h->err, h->stream)) {
            prof_end(h, LRU_PROF_FLUSH);
            return LRU_ERR_UNSUPPORTED;
        }
        if (h->pf) {
            launch_skew_project(h->W, h->n_uni, (double*)h->G, Z.go, h->stream);
            h->launches += 1;
        }
    } else if (h->flush == LRU_FLUSH_DF) {
        launch_flush_df(h->pf, L, h->state<double>(), force, h->stream);
    } else if (h->flush != LRU_FLUSH_NATIVE) {
        if (force) LRU_DISPATCH(h, { launch_zero_split_tail<T>(L, h->state<T>(), force, h->stream); });
        if (!launch_flush_tc(h->flush, h->pf, L, (double*)h->G, h->P32h, h->P32l, h->Q32h, h->Q32l, h->tau,
                             force, h->err, h->stream))
            return LRU_ERR_UNSUPPORTED;
    } else {
        LRU_DISPATCH(h, { launch_flush_native<T>(h->pf, L, h->state<T>(), force, h->n_max, h->stream); });
    }
    prof_end(h, LRU_PROF_FLUSH);
    LRU_DISPATCH(h, { launch_flush_finish<T>(L, h->state<T>(), force, h->stream); });
    return cuda_check();
}

lru_status lru_accept(lru_handle h, const uint8_t* mask) {
    LRU_RANGE();
    if (!h) return LRU_ERR_ARG;
    if (!h->has_prop) return LRU_ERR_STATE;
    CK(cudaSetDevice(h->device));
    DevLayout L = h->layout();
    // the delayed Pfaffian wrote both slots at propose time: no pass over A_0^{-1}
    const int nitems = (h->pf && h->delayed) ? 0 : h->nitems;
    h->launches += (nitems > 0 ? 1 : 0) + 1;
    prof_begin(h, LRU_PROF_ACCEPT);
    LRU_DISPATCH(h, {
        launch_accept<T>(h->pf, h->delayed, h->df, L, h->state<T>(), h->lastV, mask, h->d_items, nitems, h->stream);
    });
    prof_end(h, LRU_PROF_ACCEPT);
    lru_status s = cuda_check();
    if (s != LRU_OK) return s;
    if (h->delayed) return do_flush(h, nullptr);
    return LRU_OK;
}

lru_status lru_flush_delayed(lru_handle h, const uint8_t* mask) {
    LRU_RANGE();
    if (!h) return LRU_ERR_ARG;
    if (!h->delayed) return LRU_OK;
    CK(cudaSetDevice(h->device));
    if (!mask) {
        // all walkers: a device mask of ones
        uint8_t* ones = nullptr;
        CK(cudaMallocAsync((void**)&ones, h->W, h->stream));
        CK(cudaMemsetAsync(ones, 1, h->W, h->stream));
        lru_status s = do_flush(h, ones);
        cudaFreeAsync(ones, h->stream);
        return s;
    }
    return do_flush(h, mask);
}

lru_status lru_get_inverse(lru_handle h, void* out) {
    LRU_RANGE();
    if (!h || !out) return LRU_ERR_ARG;
    CK(cudaSetDevice(h->device));
    DevLayout L = h->layout();
    h->launches += 1;
    LRU_DISPATCH(h, { launch_get_inverse<T>(h->pf, h->delayed, L, h->state<T>(), (T*)out, h->stream); });
    return cuda_check();
}

lru_status lru_get_logvalue(lru_handle h, double* logabs, void* sign) {
    LRU_RANGE();
    if (!h) return LRU_ERR_ARG;
    CK(cudaSetDevice(h->device));
    if (logabs) CK(cudaMemcpyAsync(logabs, h->logabs, h->W * sizeof(double), cudaMemcpyDefault, h->stream));
    if (sign) CK(cudaMemcpyAsync(sign, h->sgn, h->W * dtype_size(h->dtype), cudaMemcpyDefault, h->stream));
    return LRU_OK;
}

lru_status lru_get_delay(lru_handle h, int32_t* tau) {
    LRU_RANGE();
    if (!h || !tau) return LRU_ERR_ARG;
    CK(cudaSetDevice(h->device));
    CK(cudaMemcpyAsync(tau, h->tau, h->W * sizeof(int), cudaMemcpyDefault, h->stream));
    return LRU_OK;
}

lru_status lru_state_bytes(lru_handle h, size_t* bytes) {
    LRU_RANGE();
    if (!h || !bytes) return LRU_ERR_ARG;
    *bytes = h->persist_bytes;
    return LRU_OK;
}

lru_status lru_save_state(lru_handle h, void* buf) {
    LRU_RANGE();
    if (!h || !buf) return LRU_ERR_ARG;
    CK(cudaSetDevice(h->device));
    CK(cudaMemcpyAsync(buf, h->base, h->persist_bytes, cudaMemcpyDefault, h->stream));
    return LRU_OK;
}

lru_status lru_load_state(lru_handle h, const void* buf) {
    LRU_RANGE();
    if (!h || !buf) return LRU_ERR_ARG;
    CK(cudaSetDevice(h->device));
    CK(cudaMemcpyAsync(h->base, buf, h->persist_bytes, cudaMemcpyDefault, h->stream));
    h->has_prop = false;
    return LRU_OK;
}

lru_status lru_check_device_error(lru_handle h) {
    LRU_RANGE();
    if (!h) return LRU_ERR_ARG;
    CK(cudaSetDevice(h->device));
    CK(cudaStreamSynchronize(h->stream));
    int e = 0;
    CK(cudaMemcpy(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) CK(cudaMemset(h->err, 0, sizeof(int)));
#ifdef LRU_DEBUG
    // the guard zones must still hold their pattern: a write past the end of a
    // region of the state (or of the scratch) lands in one of them
    std::vector<unsigned char> guard(CANARY_BYTES);
    for (size_t c : h->canaries) {
        CK(cudaMemcpy(guard.data(), h->base + c, CANARY_BYTES, cudaMemcpyDeviceToHost));
        for (unsigned char v : guard)
            if (v != 0xA5 && !e) e = DEV_ERR_CANARY;
    }
#endif
    if (e == DEV_ERR_TIMEOUT) return LRU_ERR_TIMEOUT;
    if (e) return LRU_ERR_CUDA;
    return LRU_OK;
}

lru_status lru_wait_selftest(lru_handle h, int64_t polls) {
    LRU_RANGE();
    if (!h || polls < 0 || polls > (1ll << 24)) return LRU_ERR_ARG;
    CK(cudaSetDevice(h->device));
    CK(cudaMemsetAsync(h->d_never, 0, sizeof(int), h->stream));
    h->launches += 1;
    launch_wait_selftest(h->d_never, (long long)polls, h->err, h->stream);
    return cuda_check();
}

lru_status lru_form_row_moves(lru_handle h, const void* Phi, int32_t m, const int32_t* occ, const int32_t* slot,
                              const int32_t* new_row, void* V_out, int32_t* idx_out) {
    LRU_RANGE();
    if (!h || !Phi || !occ || !slot || !new_row || !V_out || !idx_out || m < 1) return LRU_ERR_ARG;
    if (h->pf || h->n_uni <= 0) return LRU_ERR_ARG;
    CK(cudaSetDevice(h->device));
    DevLayout L = h->layout();
    h->launches += 1;
    LRU_DISPATCH(h, {
        launch_form_row_moves<T>(L, (const T*)Phi, m, occ, slot, new_row, (T*)V_out, idx_out, h->stream);
    });
    return cuda_check();
}

lru_status lru_form_pf_moves(lru_handle h, const void* F, int32_t m, const int32_t* pos, const int32_t* slot,
                             const int32_t* new_site, void* B_out, int32_t* idx_out) {
    LRU_RANGE();
    if (!h || !F || !pos || !slot || !new_site || !B_out || !idx_out || m < 1) return LRU_ERR_ARG;
    if (!h->pf || h->n_uni <= 0 || (h->kk != 2 && h->kk != 4) || h->d_kv) return LRU_ERR_ARG;
    CK(cudaSetDevice(h->device));
    DevLayout L = h->layout();
    h->launches += 1;
    LRU_DISPATCH(h, {
        launch_form_pf_moves<T>(L, (const T*)F, m, pos, slot, new_site, (T*)B_out, idx_out, h->stream);
    });
    return cuda_check();
}

lru_status lru_commit_moves(lru_handle h, int32_t* occ, const int32_t* slot, const int32_t* new_row,
                            const uint8_t* mask) {
    LRU_RANGE();
    if (!h || !occ || !slot || !new_row) return LRU_ERR_ARG;
    if (h->n_uni <= 0) return LRU_ERR_ARG;
    CK(cudaSetDevice(h->device));
    h->launches += 1;
    launch_commit_moves(h->W, h->n_uni, h->pf ? h->kk / 2 : h->kk, occ, slot, new_row, mask, h->pst, h->stream);
    return cuda_check();
}

lru_status lru_gather_rows(lru_handle h, const void* Phi, int32_t m, const int32_t* occ, void* A_out) {
    LRU_RANGE();
    if (!h || !Phi || !occ || !A_out || m < 1) return LRU_ERR_ARG;
    if (h->n_uni <= 0) return LRU_ERR_ARG;
    CK(cudaSetDevice(h->device));
    DevLayout L = h->layout();
    h->launches += 1;
    LRU_DISPATCH(h, { launch_gather<T>(false, L, (const T*)Phi, m, occ, (T*)A_out, h->err, h->stream); });
    return cuda_check();
}

lru_status lru_gather_pairs(lru_handle h, const void* F, int32_t m, const int32_t* pos, void* A_out) {
    LRU_RANGE();
    if (!h || !F || !pos || !A_out || m < 1) return LRU_ERR_ARG;
    if (h->n_uni <= 0) return LRU_ERR_ARG;
    CK(cudaSetDevice(h->device));
    DevLayout L = h->layout();
    h->launches += 1;
    LRU_DISPATCH(h, { launch_gather<T>(true, L, (const T*)F, m, pos, (T*)A_out, h->err, h->stream); });
    return cuda_check();
}

lru_status lru_log_ratio(lru_handle h, void* logr) {
    LRU_RANGE();
    if (!h || !logr) return LRU_ERR_ARG;
    if (!h->has_prop) return LRU_ERR_STATE;
    CK(cudaSetDevice(h->device));
    h->launches += 1;
    LRU_DISPATCH(h, { launch_log_ratio<T>(h->W, (const T*)h->ratio, (T*)logr, h->stream); });
    return cuda_check();
}

static lru_status do_backward(lru_handle h, bool pf, const void* g, void* gU, void* gV, void* gA, void* gC) {
    if (!h || !g) return LRU_ERR_ARG;
    if (h->pf != pf) return LRU_ERR_STATE;
    if (!h->has_prop) return LRU_ERR_STATE;
    CK(cudaSetDevice(h->device));
    if (!h->bws) {
        if (cudaMalloc(&h->bws, (size_t)2 * h->sum_n * h->kk * dtype_size(h->dtype)) != cudaSuccess) {
            cudaGetLastError();
            h->bws = nullptr;
            return LRU_ERR_NOMEM;
        }
    }
    DevLayout L = h->layout();
    h->launches += 1;
    LRU_DISPATCH(h, {
        launch_backward<T>(pf, h->delayed, L, h->state<T>(), h->lastV, (const T*)h->lastC, (const T*)g, (T*)h->bws,
                           (T*)gU, (T*)gV, (T*)gA, (T*)gC, h->stream);
    });
    return cuda_check();
}

lru_status lru_backward_det(lru_handle h, const void* g, void* gU, void* gV, void* gA) {
    LRU_RANGE();
    return do_backward(h, false, g, gU, gV, gA, nullptr);
}

lru_status lru_backward_pf(lru_handle h, const void* g, void* gB, void* gC, void* gA) {
    LRU_RANGE();
    return do_backward(h, true, g, gB, nullptr, gA, gC);
}

lru_status lru_backward_logvalue(lru_handle h, const void* g, void* gA) {
    LRU_RANGE();
    if (!h || !g || !gA) return LRU_ERR_ARG;
    CK(cudaSetDevice(h->device));
    DevLayout L = h->layout();
    h->launches += 1;
    LRU_DISPATCH(h, { launch_backward_logvalue<T>(h->pf, h->delayed, L, h->state<T>(), (const T*)g, (T*)gA, h->stream); });
    return cuda_check();
}

lru_status lru_scatter_rows_add(lru_handle h, const void* gA, const int32_t* rows, int32_t m, void* gPhi) {
    LRU_RANGE();
    if (!h || !gA || !rows || !gPhi || m < 1) return LRU_ERR_ARG;
    if (h->n_uni <= 0) return LRU_ERR_ARG;
    CK(cudaSetDevice(h->device));
    DevLayout L = h->layout();
    h->launches += 1;
    LRU_DISPATCH(h, { launch_scatter_rows<T>(L, (const T*)gA, rows, m, (T*)gPhi, h->err, h->stream); });
    return cuda_check();
}

lru_status lru_profile_enable(lru_handle h, int32_t on) {
    LRU_RANGE();
    if (!h) return LRU_ERR_ARG;
    h->prof_on = on != 0;
    return LRU_OK;
}

lru_status lru_profile_read(lru_handle h, int32_t cls, double* total_ms, int64_t* launches) {
    LRU_RANGE();
    if (!h || cls < 0 || cls >= LRU_PROF_CLASSES) return LRU_ERR_ARG;
    CK(cudaSetDevice(h->device));
    CK(cudaStreamSynchronize(h->stream));
    double t = 0.0;
    const size_t used = h->prof_used[cls];
    for (size_t i = 0; i < used; ++i) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, h->prof_ev[cls][i].first, h->prof_ev[cls][i].second));
        t += ms;
    }
    h->prof_used[cls] = 0;
    if (total_ms) *total_ms = t;
    if (launches) *launches = (int64_t)used;
    return LRU_OK;
}

lru_status lru_launch_count(lru_handle h, int64_t* count) {
    LRU_RANGE();
    if (!h || !count) return LRU_ERR_ARG;
    *count = h->launches;
    return LRU_OK;
}

static lru_status batched_dense(bool pf, int32_t dtype, int64_t W, int32_t n, const void* A, double* logabs,
                                void* sign, void* stream) {
    if (W < 1 || W > (int64_t)INT32_MAX || n < 1 || n > MAXN || !A || !logabs || !sign || dtype_size(dtype) == 0)
        return LRU_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 148;
    CK(cudaGetDevice(&dev));
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) { cudaGetLastError(); nsm = 148; }
    const int nws = (int)std::min<int64_t>(W, 2 * nsm);
    void* ws = nullptr;
    CK(cudaMallocAsync(&ws, (size_t)nws * n * n * dtype_size(dtype), st));
    lru_ctx tmp;
    tmp.dtype = dtype;
    DevLayout L{};
    L.W = (int)W;
    L.n_uni = n;
    L.n_max = n;
    lru_ctx* h = &tmp;
    LRU_DISPATCH(h, {
        if (pf) launch_slogpf<T>(L, (const T*)A, nullptr, (T*)ws, nws, logabs, (T*)sign, st);
        else launch_slogdet<T>((int)W, n, (const T*)A, (T*)ws, nws, logabs, (T*)sign, st);
    });
    lru_status s = cuda_check();
    cudaFreeAsync(ws, st);
    return s;
}

lru_status lru_slogdet_batched(int32_t dtype, int64_t W, int32_t n, const void* A, double* logabs, void* sign,
                               void* stream) {
    LRU_RANGE();
    return batched_dense(false, dtype, W, n, A, logabs, sign, stream);
}

static lru_status slog_backward(bool pf, int32_t dtype, int64_t W, int32_t n, const void* A, const double* g_logabs,
                                const void* g_sign, const void* sign, void* gA, void* stream) {
    if (W < 1 || W > (int64_t)INT32_MAX || n < 1 || n > MAXN || !A || !gA || dtype_size(dtype) == 0) return LRU_ERR_ARG;
    if (pf && (n & 1)) return LRU_ERR_ARG;
    if (g_sign && !sign) return LRU_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 148;
    CK(cudaGetDevice(&dev));
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) { cudaGetLastError(); nsm = 148; }
    const int nws = (int)std::min<int64_t>(W, 2 * nsm);
    const size_t sz = dtype_size(dtype), nn = (size_t)n * n;
    // the inverses (W n^2), the Gauss-Jordan slots (nws n^2) and the per-walker status
    void* buf = nullptr;
    CK(cudaMallocAsync(&buf, align_up((size_t)W * nn * sz) + align_up((size_t)nws * nn * sz) + (size_t)W * sizeof(int),
                       st));
    unsigned char* b = (unsigned char*)buf;
    void* Ginv = b;
    void* ws = b + align_up((size_t)W * nn * sz);
    int* pst = (int*)(b + align_up((size_t)W * nn * sz) + align_up((size_t)nws * nn * sz));
    DevLayout L{};
    L.W = (int)W;
    L.n_uni = n;
    L.n_max = n;
    L.kk = 1;
    lru_ctx tmp;
    tmp.dtype = dtype;
    lru_ctx* h = &tmp;
    LRU_DISPATCH(h, {
        DevState<T> S{};
        S.G = (T*)Ginv;
        S.pst = pst;
        launch_refresh<T>(false, false, L, S, (const T*)A, nullptr, (T*)ws, nws, nullptr, false, st);
        launch_slog_grad<T>((int)W, n, pf, (const T*)Ginv, g_logabs, (const T*)g_sign, (const T*)sign, (T*)gA, st);
    });
    lru_status s = cuda_check();
    cudaFreeAsync(buf, st);
    return s;
}

lru_status lru_slogdet_backward(int32_t dtype, int64_t W, int32_t n, const void* A, const double* g_logabs,
                                const void* g_sign, const void* sign, void* gA, void* stream) {
    LRU_RANGE();
    return slog_backward(false, dtype, W, n, A, g_logabs, g_sign, sign, gA, stream);
}

lru_status lru_slogpf_backward(int32_t dtype, int64_t W, int32_t n, const void* A, const double* g_logabs,
                               const void* g_sign, const void* sign, void* gA, void* stream) {
    LRU_RANGE();
    return slog_backward(true, dtype, W, n, A, g_logabs, g_sign, sign, gA, stream);
}

lru_status lru_slogpf_batched(int32_t dtype, int64_t W, int32_t n, const void* A, double* logabs, void* sign,
                              void* stream) {
    LRU_RANGE();
    if (n & 1) return LRU_ERR_ARG;
    return batched_dense(true, dtype, W, n, A, logabs, sign, stream);
}

}  // extern "C"
