// common.cuh -- shared host/device helpers of libodp (status, scratch, SM
// count, small warp/block primitives).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "odp.h"

#define ODP_FULL_MASK 0xFFFFFFFFu

namespace odp {

// ------------------------------------------------------------------ host

// Scratch blocks are cached per (device, stream, slot) and grow on demand.
// Slots keep the fingerprint and analysis scratch apart.
enum ScratchSlot {
    SLOT_FP_PLAN = 0,
    SLOT_AN_MAIN = 1,
    SLOT_AN_TABLE = 2,
    SLOT_AN_SORT = 3,
    SLOT_AN_SITES = 4,
    SLOT_SERVE = 5,
    SLOT_FP_LOG = 6,
    SLOT_COUNT = 8
};

// Returns a device block of at least `bytes` bytes for (current device,
// stream, slot), or null with *status = ODP_ERR_OOM.  *fresh (if given) is
// set when the block was just allocated (its contents are undefined).
void* scratch_get(int slot, size_t bytes, cudaStream_t stream, int* status,
                  bool* fresh = nullptr);

// Frees the (current device, stream, slot) block (stream-ordered).
void release_slot(int slot, cudaStream_t stream);

// Size of the block scratch_get allocates for a request of `bytes` (it keeps
// a quarter of headroom, so slightly larger later requests reuse the block).
size_t scratch_block_bytes(size_t bytes);

// Device scratch of one odp_fingerprint call over n buffers: the block its
// plan (tile and node offsets, tree counters, subtree roots) takes.
size_t fp_plan_scratch_bytes(uint64_t n);

int device_sm_count();       // SMs of the current device
int current_device();
int32_t* device_status_word(int* status);  // per-device fingerprint status

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? ODP_OK : ODP_ERR_CUDA; }

#define ODP_CHECK_CUDA(expr)                              \
    do {                                                  \
        cudaError_t _e = (expr);                          \
        if (_e != cudaSuccess) return ODP_ERR_CUDA;       \
    } while (0)

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ---------------------------------------------------------------- device

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src) {
    return __shfl_sync(ODP_FULL_MASK, v, src);
}
__device__ __forceinline__ uint64_t shfl_down64(uint64_t v, int d) {
    return __shfl_down_sync(ODP_FULL_MASK, v, d);
}

// A finding record written as three aligned 16-byte words (the record type
// is byte-packed, so a plain struct store would be split into byte stores).
// `items` must be 16-byte aligned.
__device__ __forceinline__ void store_finding(odp_finding* items, uint64_t pos, uint32_t kind,
                                              uint32_t site, uint32_t partner_site,
                                              uint64_t event, uint64_t partner,
                                              uint64_t wasted_bytes, uint64_t wasted_ns) {
    uint4* d = reinterpret_cast<uint4*>(items) + 3 * pos;
    d[0] = make_uint4(kind, site, partner_site, 0u);
    d[1] = make_uint4((uint32_t)event, (uint32_t)(event >> 32), (uint32_t)partner,
                      (uint32_t)(partner >> 32));
    d[2] = make_uint4((uint32_t)wasted_bytes, (uint32_t)(wasted_bytes >> 32),
                      (uint32_t)wasted_ns, (uint32_t)(wasted_ns >> 32));
}

// Records the first (lowest-index) device error: packs (index, code) so that
// atomicMin keeps the smallest index.  code is the negated status (1..127).
__device__ __forceinline__ void record_error(unsigned long long* word, uint64_t index, int status) {
    unsigned long long v = ((unsigned long long)index << 8) | (unsigned long long)(-status & 0xFF);
    atomicMin(word, v);
}

// Block-wide exclusive scan of one u32 per thread (blockDim.x multiple of 32,
// at most 1024).  Returns the exclusive prefix; *total gets the block sum.
__device__ __forceinline__ uint32_t block_exclusive_scan_u32(uint32_t v, uint32_t* total,
                                                             uint32_t* smem /*>=33*/) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(ODP_FULL_MASK, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) smem[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < nwarps ? smem[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(ODP_FULL_MASK, s, d);
            if (lane >= d) s += y;
        }
        if (lane < nwarps) smem[lane] = s;  // inclusive per-warp sums
        if (lane == nwarps - 1) smem[32] = s;
    }
    __syncthreads();
    uint32_t base = warp > 0 ? smem[warp - 1] : 0;
    *total = smem[32];
    uint32_t r = base + x - v;
    __syncthreads();
    return r;
}

// Programmatic dependent launch: a kernel launched with pdl() may be placed
// while the kernel before it on the stream is finishing (its launch overlaps
// the predecessor's last blocks instead of following its completion).  Its
// first statement, pdl_entry(), waits until that kernel has completed and its
// writes are visible.  No kernel triggers its successor early: the successor
// is placed as the kernel's blocks exit.  Measured on the analysis, triggering
// at entry instead let successors sit resident through the many waves of a
// 5e7-event call (3 % slower than plain launches); triggering at exit saves
// 2.5 % there and 14 % on 5e6 events.
__device__ __forceinline__ void pdl_entry() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Launches with programmatic serialization when `allow` is set, plainly
// otherwise (pdl_entry() is then a no-op).
template <typename... KArgs, typename... Args>
inline void pdl_if(bool allow, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                   cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = allow ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename... KArgs, typename... Args>
inline void pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                Args... args) {
    pdl_if(true, kernel, grid, block, smem, s, args...);
}

}  // namespace odp
