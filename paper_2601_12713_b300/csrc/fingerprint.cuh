// fingerprint.cuh -- launch schedule of the fingerprint kernels (host side).
#pragma once

#include "common.cuh"

namespace odp {

constexpr int TILE_WARPS = 8;

// Launch parameters of one odp_fingerprint call.  None of them changes a
// result: tiles are aligned power-of-two blocks of chunks, which the
// left-balanced tree combines into the same root whatever their size.
struct FpLaunch {
    int warps_per_cta = TILE_WARPS;  // 4, 8 or 16
    int ctas_per_sm = 0;             // 0: occupancy maximum
    uint32_t tmin_scale = 2;         // target tiles per buffer = scale * warps / n
    int stages = 2;                  // 0: register loads; 2 or 4: bulk-copy ring slots per warp
};

// ptrs == sizes == null with n == 1: the one buffer is (one_ptr, one_size),
// given by value from the host.
int fp_run(const void* const* ptrs, const uint64_t* sizes, uint64_t n, odp_fp128* out,
           cudaStream_t stream, const FpLaunch& L, const void* one_ptr = nullptr,
           uint64_t one_size = 0);

// Schedule for a batch of n buffers: the autotuned entry for n's size class
// if one exists, else the defaults (tile target scale 1 for a single buffer).
FpLaunch fp_schedule_for(uint64_t n);

}  // namespace odp
