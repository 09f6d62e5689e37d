// Top-k selection over caller-provided device scores that allocates no memory.
//
// Some callers cannot allocate device memory while they run: a component that has reserved all device
// memory for its own pool, or a serving loop that must not take the device-wide synchronisation that
// cudaMalloc / cudaFree imply.  This entry point serves them.  Its scratch lives in one file-scope
// __device__ array of fixed size (every GPU that loads the library holds it until the process exits),
// so a call allocates nothing: the caller passes the scores and the output buffers.
#include <mutex>

#include "internal.cuh"

namespace {

constexpr int32_t kMaxQueries = 64;   // queries per call
constexpr int32_t kMaxK = 1024;       // kmax per call
constexpr int32_t kMaxBlocks = 1024;  // per-query blocks of the radix passes (topk_blocks_per_query <= 1024)

// scratch layout, in 4-byte words: hist [Q][256], state [Q][4], tie counts [Q][kMaxBlocks],
// candidate ids [Q][kMaxK], candidate values [Q][kMaxK], query nodes [Q], query k [Q]
constexpr size_t kHistWords = (size_t)kMaxQueries * 256;
constexpr size_t kStateWords = (size_t)kMaxQueries * 4;
constexpr size_t kTieWords = (size_t)kMaxQueries * kMaxBlocks;
constexpr size_t kCandWords = (size_t)kMaxQueries * kMaxK;
constexpr size_t kScratchWords = kHistWords + kStateWords + kTieWords + 2 * kCandWords + 2 * (size_t)kMaxQueries;
constexpr size_t kScratchBytes = kScratchWords * 4;
static_assert(kScratchBytes == 853504, "scratch size documented in include/probesim.h");

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void *g_addr[256];  // device address of g_scratch per device ordinal, set up on a device's first call

bool device_memory(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

probesim_status err(probesim_status s, const char *msg) {
    ps::set_last_error(msg);
    return s;
}

}  // namespace

extern "C" probesim_status probesim_topk_select_noalloc(const float *scores, int32_t n, int32_t nq,
                                                        const int32_t *nodes, const int32_t *ks, int32_t kmax,
                                                        int32_t *ids, float *vals, void *stream) {
    ps::set_last_error("");
    if (!scores || !nodes || !ks || !ids || !vals) return err(PROBESIM_E_INVALID, "null argument");
    if (n < 2) return err(PROBESIM_E_INVALID, "n must be >= 2");
    if (nq < 1 || nq > kMaxQueries) return err(PROBESIM_E_INVALID, "nq must lie in [1, 64] (the scratch holds 64 queries)");
    if (kmax < 1 || kmax > kMaxK || kmax > n - 1)
        return err(PROBESIM_E_INVALID, "kmax must lie in [1, min(1024, n-1)] (the scratch holds 1024 candidates per query)");
    for (int32_t i = 0; i < nq; ++i) {
        if (nodes[i] < 0 || nodes[i] >= n) return err(PROBESIM_E_RANGE, "query node outside [0, n)");
        if (ks[i] < 1 || ks[i] > kmax) return err(PROBESIM_E_INVALID, "k must lie in [1, kmax]");
    }
    if (!device_memory(scores) || !device_memory(ids) || !device_memory(vals))
        return err(PROBESIM_E_INVALID, "scores, ids and vals must be device memory");
    std::lock_guard<std::mutex> lk(g_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        cudaGetLastError();
        return err(PROBESIM_E_CUDA, "cudaGetDevice failed");
    }
    if (!g_addr[dev]) {  // once per device, with that device current: the device address of the array,
        void *p = nullptr;   // and the top-k kernels loaded (module loads may allocate; later calls do not)
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return err(PROBESIM_E_CUDA, "cudaGetSymbolAddress of the scratch array failed");
        }
        if (ps::topk_preload() != cudaSuccess) {
            cudaGetLastError();
            return err(PROBESIM_E_CUDA, "loading the top-k kernels failed");
        }
        g_addr[dev] = p;
    }
    uint32_t *w = static_cast<uint32_t *>(g_addr[dev]);
    ps::TopkScratch sc;
    sc.hist = w;
    sc.state = w + kHistWords;
    sc.tiecnt = sc.state + kStateWords;
    sc.cand_id = reinterpret_cast<int32_t *>(sc.tiecnt + kTieWords);
    sc.cand_val = reinterpret_cast<float *>(sc.cand_id + kCandWords);
    int32_t *d_nodes = reinterpret_cast<int32_t *>(sc.cand_val + kCandWords);
    int32_t *d_ks = d_nodes + kMaxQueries;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(d_nodes, nodes, sizeof(int32_t) * nq, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_ks, ks, sizeof(int32_t) * nq, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        return err(PROBESIM_E_CUDA, "copy of the query arrays failed");
    }
    // the kernels write every scratch word before they read it (histograms and state are reset by the
    // first kernel), so nothing left by an earlier call is read
    ps::launch_topk(n, nq, scores, d_nodes, d_ks, kmax, sc, ids, vals, st, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        ps::set_last_error((std::string("top-k kernels failed: ") + cudaGetErrorString(e)).c_str());
        return PROBESIM_E_CUDA;
    }
    return PROBESIM_OK;
}
