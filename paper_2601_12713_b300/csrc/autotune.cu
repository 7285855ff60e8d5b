// autotune.cu -- schedule search for odp_fingerprint and its cache.
//
// A schedule (warps per CTA, CTAs per SM, tile-count target) only changes how
// the tiles are spread over the GPU, never a result; the search checks that
// every candidate reproduces the first candidate's fingerprints bit for bit.
// The best schedule is kept per size class (bit length of n), in memory and,
// when ODP_AUTOTUNE_CACHE names a file, in a small JSON file.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fingerprint.cuh"

namespace odp {
namespace {

std::mutex g_mu;
std::map<int, FpLaunch> g_cache;
bool g_loaded = false;

int size_class(uint64_t n) {
    int b = 0;
    while (n) {
        ++b;
        n >>= 1;
    }
    return b;
}

const char* cache_path() { return std::getenv("ODP_AUTOTUNE_CACHE"); }

// {"fp": {"<class>": [warps, ctas, tmin_scale, stages], ...}}
void load_locked(const char* path) {
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    std::string text;
    char buf[4096];
    size_t k;
    while ((k = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, k);
    std::fclose(f);
    const char* p = std::strstr(text.c_str(), "\"fp\"");
    if (!p) return;
    while ((p = std::strchr(p, '"')) != nullptr) {
        int cls, w, c, t, st = 0;
        if (std::sscanf(p, "\"%d\": [%d, %d, %d, %d]", &cls, &w, &c, &t, &st) >= 4) {
            FpLaunch L;
            L.warps_per_cta = w;
            L.ctas_per_sm = c;
            L.tmin_scale = (uint32_t)std::max(1, t);
            L.stages = st;
            g_cache[cls] = L;
        }
        ++p;
    }
}

void save_locked(const char* path) {
    FILE* f = std::fopen(path, "w");
    if (!f) return;
    std::fprintf(f, "{\"fp\": {");
    bool first = true;
    for (auto& kv : g_cache) {
        std::fprintf(f, "%s\"%d\": [%d, %d, %u, %d]", first ? "" : ", ", kv.first,
                     kv.second.warps_per_cta, kv.second.ctas_per_sm, kv.second.tmin_scale,
                     kv.second.stages);
        first = false;
    }
    std::fprintf(f, "}}\n");
    std::fclose(f);
}

void ensure_loaded_locked() {
    if (g_loaded) return;
    g_loaded = true;
    if (const char* p = cache_path()) load_locked(p);
}

FpLaunch from_public(const odp_fp_schedule& s) {
    FpLaunch L;
    L.warps_per_cta = s.warps_per_cta;
    L.ctas_per_sm = s.ctas_per_sm;
    L.tmin_scale = (uint32_t)std::max(1, s.tmin_scale);
    L.stages = s.load_stages;
    return L;
}

odp_fp_schedule to_public(const FpLaunch& L) {
    odp_fp_schedule s;
    s.warps_per_cta = L.warps_per_cta;
    s.ctas_per_sm = L.ctas_per_sm;
    s.tmin_scale = (int32_t)L.tmin_scale;
    s.load_stages = L.stages;
    return s;
}

}  // namespace

FpLaunch fp_schedule_for(uint64_t n) {
    std::lock_guard<std::mutex> lk(g_mu);
    ensure_loaded_locked();
    auto it = g_cache.find(size_class(n));
    if (it != g_cache.end()) return it->second;
    FpLaunch L;
    // one buffer: about one tile per warp (static first tiles, least climbing)
    if (n == 1) L.tmin_scale = 1;
    return L;
}

}  // namespace odp

extern "C" {

int odp_fingerprint_with(const odp_fp_schedule* sched, const void* const* ptrs,
                         const uint64_t* sizes, uint64_t n, odp_fp128* out128,
                         cudaStream_t stream) {
    if (!sched) return ODP_ERR_INVALID_ARG;
    if (n > 0 && (!ptrs || !sizes)) return ODP_ERR_INVALID_ARG;
    if (sched->warps_per_cta != 4 && sched->warps_per_cta != 8 && sched->warps_per_cta != 16)
        return ODP_ERR_INVALID_ARG;
    if (sched->ctas_per_sm < 0 || sched->tmin_scale < 1) return ODP_ERR_INVALID_ARG;
    if (sched->load_stages != 0 && sched->load_stages != 2 && sched->load_stages != 4)
        return ODP_ERR_INVALID_ARG;
    if (sched->warps_per_cta == 16 && sched->load_stages == 4) return ODP_ERR_INVALID_ARG;
    return odp::fp_run(ptrs, sizes, n, out128, stream, odp::from_public(*sched));
}

int odp_autotune_fingerprint(const void* const* ptrs, const uint64_t* sizes, uint64_t n,
                             odp_fp128* out128, cudaStream_t stream, int reps,
                             odp_fp_schedule* best, float* best_ms) {
    if (n == 0) return ODP_OK;
    if (!ptrs || !sizes || !out128) return ODP_ERR_INVALID_ARG;
    if (reps < 1) reps = 3;
    std::vector<odp::FpLaunch> cand;
    for (int w : {4, 8, 16})
        for (int st : {0, 2, 4})
            for (uint32_t t : {1u, 2u, 4u, 16u}) {
                if (w == 16 && st == 4) continue;
                odp::FpLaunch L;
                L.warps_per_cta = w;
                L.tmin_scale = t;
                L.stages = st;
                cand.push_back(L);
            }
    std::vector<odp_fp128> ref((size_t)n), cur((size_t)n);
    cudaEvent_t e0, e1;
    ODP_CHECK_CUDA(cudaEventCreate(&e0));
    ODP_CHECK_CUDA(cudaEventCreate(&e1));
    float best_t = 1e30f;
    odp::FpLaunch best_L;
    int rc = ODP_OK;
    for (size_t c = 0; c < cand.size() && rc == ODP_OK; ++c) {
        rc = odp::fp_run(ptrs, sizes, n, out128, stream, cand[c]);  // warm-up
        if (rc != ODP_OK) break;
        cudaEventRecord(e0, stream);
        for (int r = 0; r < reps && rc == ODP_OK; ++r)
            rc = odp::fp_run(ptrs, sizes, n, out128, stream, cand[c]);
        cudaEventRecord(e1, stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = ODP_ERR_CUDA;
        if (rc != ODP_OK) break;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        auto& dst = c == 0 ? ref : cur;
        if (cudaMemcpy(dst.data(), out128, n * sizeof(odp_fp128), cudaMemcpyDeviceToHost) !=
            cudaSuccess) {
            rc = ODP_ERR_CUDA;
            break;
        }
        if (c > 0 && std::memcmp(ref.data(), cur.data(), n * sizeof(odp_fp128)) != 0) {
            rc = ODP_ERR_MISMATCH;
            break;
        }
        if (ms < best_t) {
            best_t = ms;
            best_L = cand[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != ODP_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(odp::g_mu);
        odp::ensure_loaded_locked();
        odp::g_cache[odp::size_class(n)] = best_L;
        if (const char* p = odp::cache_path()) odp::save_locked(p);
    }
    if (best) *best = odp::to_public(best_L);
    if (best_ms) *best_ms = best_t;
    // leave the fingerprints of the chosen schedule in out128
    return odp::fp_run(ptrs, sizes, n, out128, stream, best_L);
}

int odp_autotune_clear(void) {
    std::lock_guard<std::mutex> lk(odp::g_mu);
    odp::g_cache.clear();
    odp::g_loaded = true;
    return ODP_OK;
}

}  // extern "C"
