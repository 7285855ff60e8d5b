// runtime.cu -- allocator hook, scratch cache, device status words and the
// status-string table of libodp.
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace odp {
namespace {

struct Block {
    void* ptr = nullptr;
    size_t bytes = 0;
};

struct Allocator {
    odp_alloc_fn alloc = nullptr;
    odp_free_fn free = nullptr;
    void* ctx = nullptr;
};

std::mutex g_mu;
Allocator g_alloc;
std::map<std::tuple<int, cudaStream_t, int>, Block> g_blocks;
std::map<int, int32_t*> g_status_words;
std::map<int, int> g_sm_count;

void* raw_alloc(size_t bytes, cudaStream_t s) {
    if (g_alloc.alloc) return g_alloc.alloc(bytes, s, g_alloc.ctx);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void raw_free(void* p, cudaStream_t s) {
    if (!p) return;
    if (g_alloc.free) {
        g_alloc.free(p, s, g_alloc.ctx);
        return;
    }
    cudaFreeAsync(p, s);
}

void release_all_locked() {
    cudaDeviceSynchronize();
    for (auto& kv : g_blocks) {
        int dev = std::get<0>(kv.first);
        cudaSetDevice(dev);
        raw_free(kv.second.ptr, std::get<1>(kv.first));
    }
    g_blocks.clear();
    cudaDeviceSynchronize();
}

}  // namespace

int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

int device_sm_count() {
    int d = current_device();
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_sm_count.find(d);
    if (it != g_sm_count.end()) return it->second;
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d);
    if (n <= 0) n = 1;
    g_sm_count[d] = n;
    return n;
}

size_t scratch_block_bytes(size_t bytes) {
    return align_up(bytes < 4096 ? 4096 : bytes + bytes / 4, 1 << 16);
}

void* scratch_get(int slot, size_t bytes, cudaStream_t stream, int* status, bool* fresh) {
    int d = current_device();
    std::lock_guard<std::mutex> lk(g_mu);
    Block& b = g_blocks[std::make_tuple(d, stream, slot)];
    if (fresh) *fresh = false;
    if (b.ptr && b.bytes >= bytes) return b.ptr;
    if (fresh) *fresh = true;
    if (b.ptr) raw_free(b.ptr, stream);  // stream-ordered after earlier uses
    b.ptr = nullptr;
    b.bytes = 0;
    size_t want = scratch_block_bytes(bytes);
    void* p = raw_alloc(want, stream);
    if (!p) {
        *status = ODP_ERR_OOM;
        return nullptr;
    }
    b.ptr = p;
    b.bytes = want;
    return p;
}

void release_slot(int slot, cudaStream_t stream) {
    int d = current_device();
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_blocks.find(std::make_tuple(d, stream, slot));
    if (it == g_blocks.end()) return;
    raw_free(it->second.ptr, stream);
    g_blocks.erase(it);
}

int32_t* device_status_word(int* status) {
    int d = current_device();
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_status_words.find(d);
    if (it != g_status_words.end()) return it->second;
    int32_t* p = nullptr;
    if (cudaMalloc(&p, 16) != cudaSuccess) {
        cudaGetLastError();
        *status = ODP_ERR_OOM;
        return nullptr;
    }
    cudaMemset(p, 0, 16);
    g_status_words[d] = p;
    return p;
}

}  // namespace odp

extern "C" {

const char* odp_status_string(int status) {
    switch (status) {
        case ODP_OK: return "ODP_OK";
        case ODP_WARN_TRUNCATED: return "ODP_WARN_TRUNCATED";
        case ODP_ERR_INVALID_ARG: return "ODP_ERR_INVALID_ARG";
        case ODP_ERR_CUDA: return "ODP_ERR_CUDA";
        case ODP_ERR_OOM: return "ODP_ERR_OOM";
        case ODP_ERR_TIMEOUT: return "ODP_ERR_TIMEOUT";
        case ODP_ERR_MALFORMED: return "ODP_ERR_MALFORMED";
        case ODP_ERR_UNSORTED: return "ODP_ERR_UNSORTED";
        case ODP_ERR_UNSUPPORTED: return "ODP_ERR_UNSUPPORTED";
        case ODP_ERR_MISMATCH: return "ODP_ERR_MISMATCH";
        default: return "ODP_UNKNOWN_STATUS";
    }
}

int odp_set_allocator(odp_alloc_fn alloc_fn, odp_free_fn free_fn, void* ctx) {
    if ((alloc_fn == nullptr) != (free_fn == nullptr)) return ODP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(odp::g_mu);
    odp::release_all_locked();
    odp::g_alloc.alloc = alloc_fn;
    odp::g_alloc.free = free_fn;
    odp::g_alloc.ctx = ctx;
    return ODP_OK;
}

int odp_release_scratch(void) {
    std::lock_guard<std::mutex> lk(odp::g_mu);
    odp::release_all_locked();
    return ODP_OK;
}

int odp_fingerprint_status(cudaStream_t stream, int32_t* status) {
    if (!status) return ODP_ERR_INVALID_ARG;
    int st = ODP_OK;
    int32_t* w = odp::device_status_word(&st);
    if (!w) return st;
    int32_t h = 0;
    ODP_CHECK_CUDA(cudaMemcpyAsync(&h, w, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    ODP_CHECK_CUDA(cudaMemsetAsync(w, 0, sizeof(int32_t), stream));
    ODP_CHECK_CUDA(cudaStreamSynchronize(stream));
    *status = h;
    return ODP_OK;
}

}  // extern "C"
