// prims.cuh -- device-wide primitives for the analysis pipeline: exclusive
// scan of u32, stable LSD radix sort of (u32 key, u32 value) pairs, and an
// open-addressing table of 128-bit keys keeping the minimum u32 value.
//
// Lengths that are only known on the device are passed as pointers; grids
// are sized from a host-side upper bound and blocks past the device length
// exit at once.
#pragma once

#include <algorithm>
#include <atomic>

#include "common.cuh"

namespace odp {
namespace prim {
// Every translation unit that includes this header gets its own copy of the
// kernels (internal linkage).
namespace {

constexpr uint32_t NONE32 = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t dev_len(const uint32_t* n_dev, uint32_t n_max) {
    return n_dev ? min(*n_dev, n_max) : n_max;
}

// ------------------------------------------------------------------ scan

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 16;  // consecutive items per thread, moved as four 16-byte words
constexpr uint32_t SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Single-pass exclusive scan with decoupled look-back: blocks take tiles from
// a counter in order, publish each tile's sum ("aggregate"), then walk back
// over their predecessors' published words, 32 at a time (one per lane),
// adding aggregates until a predecessor that already published its
// inclusive prefix; then publish their own inclusive prefix.  A block only
// waits on tiles handed out before its own, which are held by running
// blocks, so every wait ends; each wait is also bounded (SCAN_WAIT_LIMIT
// polls, then *fault is set and the scan goes on with a wrong prefix, never a
// hang).
//
// tmp (u32 words, zero before its first use; every scan leaves it ready for
// the next): [0] tile counter, [1] finished blocks, [2] epoch, [3] unused,
// then one u64 per tile: epoch (30 bits) | flag (2 bits: 1 aggregate,
// 2 inclusive) | value (32 bits).  The last block out resets the counters and
// advances the epoch, so words of earlier scans never look current (also
// when a captured graph replays the same launch).
constexpr uint32_t SCAN_WAIT_LIMIT = 1u << 20;

__global__ void __launch_bounds__(SCAN_THREADS, 3)
scan_chained(const uint32_t* in, uint32_t* out, const uint32_t* n_dev, uint32_t n_max,
             uint32_t* total, uint32_t* tmp, uint32_t* fault) {
    pdl_entry();
    __shared__ uint32_t sm[40];
    __shared__ uint32_t s_tile, s_prefix;
    unsigned long long* status = reinterpret_cast<unsigned long long*>(tmp + 4);
    const uint32_t n = dev_len(n_dev, n_max);
    const uint32_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    const uint32_t epoch = *(volatile uint32_t*)(tmp + 2) & 0x3FFFFFFFu;
    const unsigned long long tag = (unsigned long long)epoch << 34;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool vec = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    if (ntiles == 0 && blockIdx.x == 0 && threadIdx.x == 0 && total) *total = 0;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(tmp, 1u);
        __syncthreads();
        const uint32_t t = s_tile;
        if (t >= ntiles) break;
        const uint32_t base = t * SCAN_TILE;
        const uint32_t i0 = base + threadIdx.x * SCAN_ITEMS;
        const bool whole = vec && i0 + SCAN_ITEMS <= n;
        uint32_t v[SCAN_ITEMS], sum = 0;
        if (whole) {
            const uint4* p = reinterpret_cast<const uint4*>(in + i0);
#pragma unroll
            for (int q = 0; q < SCAN_ITEMS / 4; ++q) {
                const uint4 w = p[q];
                v[4 * q] = w.x;
                v[4 * q + 1] = w.y;
                v[4 * q + 2] = w.z;
                v[4 * q + 3] = w.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < SCAN_ITEMS; ++k) v[k] = i0 + k < n ? in[i0 + k] : 0;
        }
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) sum += v[k];
        uint32_t tot;
        uint32_t e = block_exclusive_scan_u32(sum, &tot, sm);
        if (warp == 0) {
            uint32_t prefix = 0;
            if (t == 0) {
                if (lane == 0) atomicExch(&status[0], tag | (2ull << 32) | tot);
            } else {
                if (lane == 0) atomicExch(&status[t], tag | (1ull << 32) | tot);
                bool ok = true;
                for (long long back = (long long)t - 1; back >= 0; back -= 32) {
                    const long long j = back - lane;
                    unsigned long long w = 0;
                    bool ready = j < 0;
                    if (!ready) {
                        w = __ldcv(&status[j]);
                        ready = (w >> 34) == epoch && ((w >> 32) & 3ull) != 0;
                    }
                    uint32_t polls = 0;
                    while (!__all_sync(ODP_FULL_MASK, ready)) {
                        if (++polls > SCAN_WAIT_LIMIT) {
                            ok = false;
                            break;
                        }
                        if (!ready) {
                            w = __ldcv(&status[j]);
                            ready = (w >> 34) == epoch && ((w >> 32) & 3ull) != 0;
                        }
                    }
                    if (!ok) break;
                    const bool incl = j < 0 || ((w >> 32) & 3ull) == 2ull;
                    const uint32_t val = j < 0 ? 0u : (uint32_t)w;
                    const uint32_t im = __ballot_sync(ODP_FULL_MASK, incl);
                    if (im) {
                        const int k = __ffs(im) - 1;
                        prefix += __reduce_add_sync(ODP_FULL_MASK, lane <= k ? val : 0u);
                        break;
                    }
                    prefix += __reduce_add_sync(ODP_FULL_MASK, val);
                }
                if (!ok && lane == 0 && fault) atomicOr(fault, 1u);
                if (lane == 0) atomicExch(&status[t], tag | (2ull << 32) | (uint32_t)(prefix + tot));
            }
            if (lane == 0) s_prefix = prefix;
        }
        __syncthreads();
        e += s_prefix;
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            const uint32_t x = v[k];
            v[k] = e;
            e += x;
        }
        if (whole) {
            uint4* p = reinterpret_cast<uint4*>(out + i0);
#pragma unroll
            for (int q = 0; q < SCAN_ITEMS / 4; ++q)
                p[q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else {
#pragma unroll
            for (int k = 0; k < SCAN_ITEMS; ++k)
                if (i0 + k < n) out[i0 + k] = v[k];
        }
        if (t == ntiles - 1 && threadIdx.x == 0 && total) *total = s_prefix + tot;
        __syncthreads();  // s_tile, s_prefix and sm are reused by the next tile
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(tmp + 1, 1u) == gridDim.x - 1) {  // last block out
            tmp[0] = 0;
            tmp[1] = 0;
            tmp[2] = (epoch + 1) & 0x3FFFFFFFu;
            __threadfence();
        }
    }
}

// u32 words of scan scratch for up to n_max elements.
inline size_t scan_tmp_words(uint32_t n_max) {
    return 4 + 2 * ((size_t)(n_max + SCAN_TILE - 1) / SCAN_TILE + 1);
}

// Grid for a loop over `tiles` tiles: at most `per_sm` blocks per SM.
inline uint32_t tile_grid(uint32_t tiles, int per_sm) {
    const uint32_t cap = (uint32_t)std::max(1, device_sm_count() * per_sm);
    return std::max(1u, std::min(tiles, cap));
}

// out[i] = sum of in[0..i) for i < n; *total = sum of all (may be null).
// In place (in == out) is allowed.  tmp: scan_tmp_words(n_max) words, zero
// before its first scan; fault (may be null) is set if a wait gave up.
inline void exclusive_scan(const uint32_t* in, uint32_t* out, const uint32_t* n_dev,
                           uint32_t n_max, uint32_t* total, uint32_t* tmp, cudaStream_t s,
                           uint32_t* fault = nullptr, bool allow_pdl = false) {
    if (n_max == 0) {
        if (total) cudaMemsetAsync(total, 0, 4, s);
        return;
    }
    const uint32_t nb = (n_max + SCAN_TILE - 1) / SCAN_TILE;
    pdl_if(allow_pdl, scan_chained, tile_grid(nb, 3), SCAN_THREADS, 0, s, in, out,
           n_dev, n_max, total, tmp, fault);
}

// ------------------------------------------------------------ radix sort

constexpr int SORT_THREADS = 256;
constexpr int SORT_ROUNDS = 16;
constexpr uint32_t SORT_TILE = SORT_THREADS * SORT_ROUNDS;  // 4096 items per tile

// The digit layout of a sort by the low `key_bits` bits: an even number of
// passes (the data ends where it started), at most 8 bits each, the bits
// split evenly.  With a device-side bound on the keys (key_max, may be null)
// the device takes only the bits the bound needs, so some of the passes the
// host launched for key_bits do nothing.  The host and the device compute it
// the same way.
struct SortPass {
    int shift, bits;
    bool active;
};

__host__ __device__ __forceinline__ int sort_passes(int key_bits) {
    const int passes = (key_bits + 7) / 8;
    return passes + (passes & 1);
}

__host__ __device__ __forceinline__ SortPass sort_pass(int p, int key_bits) {
    const int npass = sort_passes(key_bits);
    SortPass r{0, 0, p < npass};
    if (!r.active) return r;
    const int per = (key_bits + npass - 1) / npass;
    for (int q = 0;; ++q) {
        int b = key_bits - r.shift;
        b = b < per ? b : per;
        r.bits = b > 1 ? b : 1;
        if (q == p) return r;
        r.shift += r.bits;
    }
}

__device__ __forceinline__ SortPass sort_pass_dev(int p, int key_bits, const uint32_t* key_max) {
    if (key_max) {
        const int need = 32 - __clz(*key_max);
        if (need < key_bits) key_bits = need;
    }
    return sort_pass(p, key_bits);
}

// Tiles of the device length n: ntd = ceil(n / SORT_TILE).  Histograms are
// stored digit-major over the device tile count, hist[d * ntd + tile], so
// the scan between the sweeps covers radix * ntd words (written to *hlen).
__device__ __forceinline__ uint32_t sort_tiles(uint32_t n) { return (n + SORT_TILE - 1) / SORT_TILE; }

// Per-tile digit histograms; blocks loop over tiles.
__global__ void __launch_bounds__(SORT_THREADS)
sort_upsweep(const uint32_t* keys, const uint32_t* n_dev, uint32_t n_max, int pass, int key_bits,
             const uint32_t* key_max, uint32_t* hist, uint32_t* hlen) {
    pdl_entry();
    __shared__ uint32_t h[256];
    const SortPass sp = sort_pass_dev(pass, key_bits, key_max);
    const int shift = sp.shift;
    const uint32_t n = sp.active ? dev_len(n_dev, n_max) : 0;
    const uint32_t ntd = sort_tiles(n);
    const uint32_t radix = 1u << sp.bits;
    if (blockIdx.x == 0 && threadIdx.x == 0) *hlen = radix * ntd;
    for (uint32_t t = blockIdx.x; t < ntd; t += gridDim.x) {
        for (uint32_t d = threadIdx.x; d < radix; d += SORT_THREADS) h[d] = 0;
        __syncthreads();
        const uint32_t base = t * SORT_TILE;
        for (uint32_t i = base + threadIdx.x; i < min(base + SORT_TILE, n); i += SORT_THREADS)
            atomicAdd(&h[(keys[i] >> shift) & (radix - 1)], 1u);
        __syncthreads();
        for (uint32_t d = threadIdx.x; d < radix; d += SORT_THREADS) hist[d * ntd + t] = h[d];
        __syncthreads();
    }
}

// Stable scatter.  Warp w of a block owns items [512 w, 512 w + 512) of the
// tile and ranks them in 16 rounds of 32 (index order) against its own digit
// counters: rank = items of the digit in the warp's earlier rounds + lower
// lanes of this round (match_any); no block barrier inside the rounds.  Then
// the counters are scanned across warps and digits, items are placed in
// shared memory in digit order and written out so that each digit's run of
// the tile lands contiguously at its global start.  Blocks loop over tiles.
__global__ void __launch_bounds__(SORT_THREADS, 4)
sort_downsweep(const uint32_t* keys, const uint32_t* vals, uint32_t* keys_out,
               uint32_t* vals_out, const uint32_t* n_dev, uint32_t n_max, int pass, int key_bits,
               const uint32_t* key_max, const uint32_t* hist_scanned) {
    pdl_entry();
    const SortPass sp = sort_pass_dev(pass, key_bits, key_max);
    const int shift = sp.shift, bits = sp.bits;
    constexpr int W = SORT_THREADS / 32;
    constexpr int PER_WARP = SORT_TILE / W;  // 512 items, SORT_ROUNDS rounds of 32
    __shared__ uint32_t base_d[256];   // global start of each digit for this tile
    __shared__ uint32_t loc_d[256];    // local start of each digit in the tile
    __shared__ uint32_t wcnt[W][256];  // per-warp digit counts, then per-warp offsets
    __shared__ uint32_t ks[SORT_TILE];
    __shared__ uint32_t vs[SORT_TILE];
    __shared__ uint32_t scan_tmp[40];
    const uint32_t n = sp.active ? dev_len(n_dev, n_max) : 0;
    const uint32_t ntd = sort_tiles(n);
    const uint32_t radix = 1u << bits;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt_mask = (1u << lane) - 1;
    for (uint32_t t = blockIdx.x; t < ntd; t += gridDim.x) {
        const uint32_t tile0 = t * SORT_TILE;
        const uint32_t tile_n = min(SORT_TILE, n - tile0);
        for (uint32_t d = threadIdx.x; d < 256; d += SORT_THREADS) {
            base_d[d] = d < radix ? hist_scanned[d * ntd + t] : 0;
            for (int w = 0; w < W; ++w) wcnt[w][d] = 0;
        }
        __syncthreads();
        uint32_t k_r[SORT_ROUNDS], r_r[SORT_ROUNDS / 2];  // ranks < 4096: two per word
        const uint32_t w0 = tile0 + warp * PER_WARP;
#pragma unroll
        for (int r = 0; r < SORT_ROUNDS; ++r) {
            const uint32_t i = w0 + r * 32 + lane;
            k_r[r] = i < n ? keys[i] : 0;
        }
#pragma unroll
        for (int r = 0; r < SORT_ROUNDS; ++r) {
            const uint32_t i = w0 + r * 32 + lane;
            const bool valid = i < n;
            const uint32_t d = valid ? (k_r[r] >> shift) & (radix - 1) : radix;
            const uint32_t peers = __match_any_sync(ODP_FULL_MASK, d);
            const uint32_t before = valid ? wcnt[warp][d] : 0;
            const uint32_t rank = before + __popc(peers & lt_mask);
            if (r & 1) r_r[r / 2] |= rank << 16; else r_r[r / 2] = rank;
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // per digit: exclusive scan over warps, then over digits
        uint32_t tot_d = 0;
        if (threadIdx.x < 256) {
            for (int w = 0; w < W; ++w) {
                const uint32_t c = wcnt[w][threadIdx.x];
                wcnt[w][threadIdx.x] = tot_d;
                tot_d += c;
            }
        }
        {
            uint32_t tot;
            const uint32_t e = block_exclusive_scan_u32(threadIdx.x < 256 ? tot_d : 0, &tot, scan_tmp);
            if (threadIdx.x < 256) loc_d[threadIdx.x] = e;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < SORT_ROUNDS; ++r) {
            const uint32_t i = w0 + r * 32 + lane;
            if (i < n) {
                const uint32_t d = (k_r[r] >> shift) & (radix - 1);
                const uint32_t pos = loc_d[d] + wcnt[warp][d] + ((r_r[r / 2] >> (16 * (r & 1))) & 0xFFFFu);
                ks[pos] = k_r[r];
                vs[pos] = vals[i];
            }
        }
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < tile_n; j += SORT_THREADS) {
            const uint32_t k = ks[j];
            const uint32_t d = (k >> shift) & (radix - 1);
            const uint32_t g = base_d[d] + (j - loc_d[d]);
            keys_out[g] = k;
            vals_out[g] = vs[j];
        }
        __syncthreads();  // shared arrays are reused by the next tile
    }
}

inline int bit_length(uint64_t v) {
    int b = 0;
    while (v) {
        ++b;
        v >>= 1;
    }
    return b;
}

struct SortTmp {
    uint32_t* keys_alt;
    uint32_t* vals_alt;
    uint32_t* hist;      // 256 * ntiles_max
    uint32_t* scan_tmp;  // scan_tmp_words(256 * ntiles_max), zero before first use
    uint32_t* hlen;      // one device word: histogram length of the current pass
    uint32_t* fault = nullptr;  // set if a scan's wait gave up (may be null)
    bool pdl = false;           // launch the passes with programmatic dependent launch (pdl())
};

inline size_t sort_hist_words(uint32_t n_max) {
    return 256ull * ((n_max + SORT_TILE - 1) / SORT_TILE + 1);
}

// ------------------------------------------------------ one-block sort

constexpr int SMALL_SORT_THREADS = 1024;
constexpr uint32_t SMALL_SORT_MAX = 8192;  // 8 items per thread
// dynamic shared memory of a one-block sort of up to `max_items` items
constexpr size_t small_sort_smem(uint32_t max_items) { return 4ull * max_items * 4 + 32ull * 256 * 4; }
constexpr size_t SMALL_SORT_SMEM = small_sort_smem(SMALL_SORT_MAX);

// Up to 8192 (key, value) pairs sorted stably by the low key_bits bits of
// the keys by one block, in shared memory: per 8-bit digit, warp w ranks its
// 256 items (index order: round-major, then lane) against its own digit
// counters, the counters are scanned across warps and digits, and the items
// move to the other buffer.  One launch instead of five per pass.
// MAXN (a multiple of 1,024, at most SMALL_SORT_MAX) sizes the shared-memory
// buffers: the caller launches with small_sort_smem(MAXN) bytes.
template <uint32_t MAXN = SMALL_SORT_MAX>
__device__ __forceinline__ void sort_small_body(uint32_t* keys, uint32_t* vals,
                                                const uint32_t* n_dev, uint32_t n_max,
                                                int key_bits) {
    static_assert(MAXN % SMALL_SORT_THREADS == 0 && MAXN <= SMALL_SORT_MAX, "tile size");
    constexpr int W = SMALL_SORT_THREADS / 32;
    constexpr int ROUNDS = MAXN / SMALL_SORT_THREADS;
    extern __shared__ __align__(16) uint32_t small_sm[];
    uint32_t* k0 = small_sm;
    uint32_t* v0 = k0 + MAXN;
    uint32_t* k1 = v0 + MAXN;
    uint32_t* v1 = k1 + MAXN;
    uint32_t(*cnt)[256] = reinterpret_cast<uint32_t(*)[256]>(v1 + MAXN);
    __shared__ uint32_t scan_tmp[40];
    __shared__ uint32_t dstart[256];
    const uint32_t n = min(dev_len(n_dev, n_max), MAXN);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1;
    for (uint32_t i = threadIdx.x; i < n; i += SMALL_SORT_THREADS) {
        k0[i] = keys[i];
        v0[i] = vals[i];
    }
    for (int shift = 0; shift < key_bits; shift += 8) {
        const int bits = min(8, key_bits - shift);
        const uint32_t radix = 1u << bits;
        for (int d = lane; d < 256; d += 32) cnt[warp][d] = 0;
        __syncthreads();
        uint32_t rank[ROUNDS];
#pragma unroll
        for (int r = 0; r < ROUNDS; ++r) {
            const uint32_t i = warp * (32 * ROUNDS) + r * 32 + lane;
            const bool valid = i < n;
            const uint32_t d = valid ? (k0[i] >> shift) & (radix - 1) : 256u;
            const uint32_t peers = __match_any_sync(ODP_FULL_MASK, d);
            const uint32_t before = valid ? cnt[warp][d] : 0;
            rank[r] = before + __popc(peers & lt);
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1) cnt[warp][d] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        uint32_t tot = 0;
        if (threadIdx.x < 256) {
            for (int w = 0; w < W; ++w) {
                const uint32_t c = cnt[w][threadIdx.x];
                cnt[w][threadIdx.x] = tot;
                tot += c;
            }
        }
        uint32_t all;
        const uint32_t e = block_exclusive_scan_u32(threadIdx.x < 256 ? tot : 0, &all, scan_tmp);
        if (threadIdx.x < 256) dstart[threadIdx.x] = e;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < ROUNDS; ++r) {
            const uint32_t i = warp * (32 * ROUNDS) + r * 32 + lane;
            if (i < n) {
                const uint32_t d = (k0[i] >> shift) & (radix - 1);
                const uint32_t pos = dstart[d] + cnt[warp][d] + rank[r];
                k1[pos] = k0[i];
                v1[pos] = v0[i];
            }
        }
        __syncthreads();
        uint32_t* t = k0;
        k0 = k1;
        k1 = t;
        t = v0;
        v0 = v1;
        v1 = t;
    }
    for (uint32_t i = threadIdx.x; i < n; i += SMALL_SORT_THREADS) {
        keys[i] = k0[i];
        vals[i] = v0[i];
    }
}

__global__ void __launch_bounds__(SMALL_SORT_THREADS) sort_small(uint32_t* keys, uint32_t* vals,
                                                                 const uint32_t* n_dev,
                                                                 uint32_t n_max, int key_bits) {
    pdl_entry();
    sort_small_body(keys, vals, n_dev, n_max, key_bits);
}

inline bool sort_small_ready() {
    static std::atomic<bool> done[256] = {};
    const int dev = current_device();
    if (dev < 0 || dev >= 256) return false;
    if (!done[dev].load(std::memory_order_acquire)) {
        if (cudaFuncSetAttribute(sort_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SMALL_SORT_SMEM) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        done[dev].store(true, std::memory_order_release);
    }
    return true;
}

// Resident sort_downsweep blocks per SM (queried once per device).
inline int downsweep_per_sm() {
    static std::atomic<int> cache[256] = {};
    const int dev = current_device();
    if (dev < 0 || dev >= 256) return 4;
    if (!cache[dev].load(std::memory_order_acquire)) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, sort_downsweep, SORT_THREADS, 0) !=
                cudaSuccess || b < 1)
            b = 4;
        cache[dev].store(b, std::memory_order_release);
    }
    return cache[dev].load(std::memory_order_acquire);
}

// Stable sort of (keys, vals) by the low `key_bits` bits of the keys; the
// result ends in (keys, vals) (ping-pong through the alternates).  key_max
// (device word, may be null): an upper bound on the keys known only on the
// device; the passes it makes unnecessary return at once.
inline void radix_sort(uint32_t* keys, uint32_t* vals, const uint32_t* n_dev, uint32_t n_max,
                       int key_bits, const SortTmp& t, cudaStream_t s,
                       const uint32_t* key_max = nullptr) {
    if (n_max == 0 || key_bits <= 0) return;
    if (n_max <= SMALL_SORT_MAX && sort_small_ready()) {
        pdl_if(t.pdl, sort_small, 1, SMALL_SORT_THREADS, SMALL_SORT_SMEM, s, keys, vals, n_dev,
               n_max, key_bits);
        return;
    }
    const uint32_t ntiles = (n_max + SORT_TILE - 1) / SORT_TILE;
    const int npass = sort_passes(key_bits);
    uint32_t *k_in = keys, *v_in = vals, *k_out = t.keys_alt, *v_out = t.vals_alt;
    for (int p = 0; p < npass; ++p) {
        // (a device-side bound can split its fewer bits into wider digits)
        const uint32_t hn = (key_max ? 256u : 1u << sort_pass(p, key_bits).bits) * ntiles;
        pdl_if(t.pdl, sort_upsweep, tile_grid(ntiles, 8), SORT_THREADS, 0, s, k_in,
               n_dev, n_max, p, key_bits, key_max, t.hist, t.hlen);
        exclusive_scan(t.hist, t.hist, t.hlen, hn, nullptr, t.scan_tmp, s, t.fault, t.pdl);
        pdl_if(t.pdl, sort_downsweep, tile_grid(ntiles, downsweep_per_sm()),
               SORT_THREADS, 0, s, k_in, v_in, k_out, v_out, n_dev, n_max, p, key_bits, key_max,
               t.hist);
        std::swap(k_in, k_out);
        std::swap(v_in, v_out);
    }
}

// ---------------------------------------------------------------- table

struct __align__(16) Key128 {
    uint64_t lo, hi;
};

__device__ __forceinline__ bool key_eq(Key128 a, Key128 b) { return a.lo == b.lo && a.hi == b.hi; }

constexpr uint64_t EMPTY_KEY = ~0ull;

// One slot per 32-byte sector: the key and its value are touched by one
// random access.
struct __align__(32) Slot {
    Key128 k;
    uint32_t v;
    uint32_t pad[3];
};

struct Table {
    Slot* slots;        // capacity + 1 slots (the last one holds the all-ones key)
    uint32_t cap_max;   // power of two
    uint32_t* cap_dev;  // capacity in use (power of two, set on the device)
    __device__ __forceinline__ Key128* key_at(uint32_t s) const { return &slots[s].k; }
    __device__ __forceinline__ uint32_t* val_at(uint32_t s) const { return &slots[s].v; }
};

// Keys and values in two arrays (16 + 4 bytes a slot): a probe touches a
// 16-byte key, and the values, read back by slot after the inserts, sit in
// an array a quarter the size of the keys (mostly in L2 at the sizes used).
struct SplitTable {
    Key128* keys;       // capacity + 1 slots (the last one holds the all-ones key)
    uint32_t* vals;     // capacity + 1 values
    uint32_t cap_max;
    uint32_t* cap_dev;
    __device__ __forceinline__ Key128* key_at(uint32_t s) const { return &keys[s]; }
    __device__ __forceinline__ uint32_t* val_at(uint32_t s) const { return &vals[s]; }
};

// Keys only, 16 bytes a slot: for grouping, where the slot index is the
// group key and no value is kept.
struct KeyTable {
    Key128* keys;       // capacity + 1 slots (the last one holds the all-ones key)
    uint32_t cap_max;
    uint32_t* cap_dev;
    __device__ __forceinline__ Key128* key_at(uint32_t s) const { return &keys[s]; }
    __device__ __forceinline__ uint32_t* val_at(uint32_t) const { return nullptr; }
};

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x ^= x >> 33;
    x *= 0xFF51AFD7ED558CCDull;
    x ^= x >> 33;
    x *= 0xC4CEB9FE1A85EC53ull;
    x ^= x >> 33;
    return x;
}

__device__ __forceinline__ uint32_t table_cap(uint32_t cnt, uint32_t cap_max) {
    uint32_t cap = 1024;
    while (cap < (uint64_t)cnt + cnt / 4 && cap < cap_max) cap <<= 1;
    return cap;
}

// Set the capacity in use to the smallest power of two >= 1.25 * count (at
// least 1024, at most cap_max; load stays <= 0.8) and clear it with whole
// 32-byte slot writes.
__device__ __forceinline__ void table_clear_body(Table t, const uint32_t* count_dev,
                                                 uint32_t count_max) {
    const uint32_t cap = table_cap(dev_len(count_dev, count_max), t.cap_max);
    if (blockIdx.x == 0 && threadIdx.x == 0) *t.cap_dev = cap;
    const uint32_t stride = gridDim.x * blockDim.x;
    uint4* w = reinterpret_cast<uint4*>(t.slots);
    const uint4 empty_key = make_uint4(~0u, ~0u, ~0u, ~0u);
    const uint4 empty_val = make_uint4(NONE32, 0u, 0u, 0u);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= cap; i += stride) {
        const uint32_t slot = i == cap ? t.cap_max : i;
        w[2 * (size_t)slot] = empty_key;
        w[2 * (size_t)slot + 1] = empty_val;
    }
}

__global__ void table_clear(Table t, const uint32_t* count_dev, uint32_t count_max) {
    pdl_entry();
    table_clear_body(t, count_dev, count_max);
}

// The same for a split table: keys, then values (NONE32), 16 bytes a write.
__global__ void table_clear(SplitTable t, const uint32_t* count_dev, uint32_t count_max) {
    pdl_entry();
    const uint32_t cap = table_cap(dev_len(count_dev, count_max), t.cap_max);
    if (blockIdx.x == 0 && threadIdx.x == 0) *t.cap_dev = cap;
    const uint32_t stride = gridDim.x * blockDim.x;
    uint4* wk = reinterpret_cast<uint4*>(t.keys);
    uint4* wv = reinterpret_cast<uint4*>(t.vals);
    const uint4 ones = make_uint4(~0u, ~0u, ~0u, ~0u);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= cap; i += stride)
        wk[i == cap ? t.cap_max : i] = ones;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cap / 4; i += stride) wv[i] = ones;
    if (blockIdx.x == 0 && threadIdx.x == 0) t.vals[t.cap_max] = NONE32;
}

// The same for a key-only table (one 16-byte write per slot).
__global__ void table_clear(KeyTable t, const uint32_t* count_dev, uint32_t count_max) {
    pdl_entry();
    const uint32_t cap = table_cap(dev_len(count_dev, count_max), t.cap_max);
    if (blockIdx.x == 0 && threadIdx.x == 0) *t.cap_dev = cap;
    const uint32_t stride = gridDim.x * blockDim.x;
    uint4* w = reinterpret_cast<uint4*>(t.keys);
    const uint4 empty_key = make_uint4(~0u, ~0u, ~0u, ~0u);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= cap; i += stride)
        w[i == cap ? t.cap_max : i] = empty_key;
}

// Inserts `k` and lowers the slot's value to v; returns the slot index, or
// NONE32 if the probe sequence exhausted the table (cannot happen at <= 50%
// load).
// What a plain (non-atomic) read of a slot's key shows: PEEK_ASK (empty,
// or possibly half-written: ask the compare-and-swap), PEEK_MINE (the slot
// holds k), PEEK_OTHER (the slot holds another key for good).  Slots change
// once per table lifetime, empty -> key; a 16-byte read may pair one
// all-ones (empty) half with a half of the new key, so only a read with no
// all-ones half is taken as a complete key.  Repeated keys then find their
// slot without an atomic, and occupied slots are passed without one.
enum { PEEK_ASK = 0, PEEK_MINE = 1, PEEK_OTHER = 2 };

__device__ __forceinline__ int peek_slot(const Key128* p, Key128 k) {
    const Key128 c = *p;
    if (c.lo == EMPTY_KEY || c.hi == EMPTY_KEY) return PEEK_ASK;
    return key_eq(c, k) ? PEEK_MINE : PEEK_OTHER;
}

// Lowers a slot's value to v; values only decrease, so a plain read at or
// below v means the atomic would change nothing.
__device__ __forceinline__ void lower_to(uint32_t* p, uint32_t v) {
    if (*p > v) atomicMin(p, v);
}

__device__ __forceinline__ uint32_t table_insert_min(const Table& t, uint32_t cap, Key128 k,
                                                     uint32_t v) {
    if (k.lo == EMPTY_KEY && k.hi == EMPTY_KEY) {
        atomicMin(&t.slots[t.cap_max].v, v);
        return t.cap_max;
    }
    const uint32_t mask = cap - 1;
    uint32_t slot = (uint32_t)mix64(k.lo ^ mix64(k.hi)) & mask;
    const Key128 empty{EMPTY_KEY, EMPTY_KEY};
    for (uint32_t probe = 0; probe < cap; ++probe) {
        // slots change only once (empty -> key), always through the 16-byte CAS
        const int seen = peek_slot(&t.slots[slot].k, k);
        if (seen == PEEK_MINE) {
            lower_to(&t.slots[slot].v, v);
            return slot;
        }
        if (seen == PEEK_ASK) {
            const Key128 cur = atomicCAS(&t.slots[slot].k, empty, k);
            if (key_eq(cur, empty) || key_eq(cur, k)) {
                lower_to(&t.slots[slot].v, v);
                return slot;
            }
        }
        slot = (slot + 1) & mask;
    }
    return NONE32;
}

// Inserts `k` without touching the slot's value; returns the slot index (one
// per distinct key), or NONE32 if the probe sequence exhausted the table.
__device__ __forceinline__ uint32_t table_insert(const Table& t, uint32_t cap, Key128 k) {
    if (k.lo == EMPTY_KEY && k.hi == EMPTY_KEY) return t.cap_max;
    const uint32_t mask = cap - 1;
    uint32_t slot = (uint32_t)mix64(k.lo ^ mix64(k.hi)) & mask;
    const Key128 empty{EMPTY_KEY, EMPTY_KEY};
    for (uint32_t probe = 0; probe < cap; ++probe) {
        const int seen = peek_slot(&t.slots[slot].k, k);
        if (seen == PEEK_MINE) return slot;
        if (seen == PEEK_ASK) {
            const Key128 cur = atomicCAS(&t.slots[slot].k, empty, k);
            if (key_eq(cur, empty) || key_eq(cur, k)) return slot;
        }
        slot = (slot + 1) & mask;
    }
    return NONE32;
}

// Inserts up to B keys per thread with their compare-and-swaps in flight
// together (the probes of different keys are independent).  use[b] false:
// out[b] = NONE32.  MIN: also lower the slot's value to v[b].  PEEK: read
// each slot before the compare-and-swap (peek_slot), which pays where many
// inserts repeat a few keys (the atomics would queue on them) and costs a
// round trip where most keys are new or rarely repeated in a table far
// larger than L2.  LOWER: read the value before lowering it (lower_to),
// which spares the atomic when an earlier insert already set a smaller one.
// fresh (may be null): set for the inserts whose compare-and-swap put the
// key into its slot (one per distinct key, except the all-ones key, which is
// never marked).
template <int B, bool MIN, bool PEEK, bool LOWER, class TableT>
__device__ __forceinline__ void table_insert_batch(const TableT& t, uint32_t cap, const Key128* k,
                                                   const uint32_t* v, const bool* use,
                                                   uint32_t* out, bool* fresh = nullptr) {
    const uint32_t mask = cap - 1;
    const Key128 empty{EMPTY_KEY, EMPTY_KEY};
    uint32_t slot[B];
    bool done[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        out[b] = NONE32;
        if (fresh) fresh[b] = false;
        done[b] = !use[b];
        slot[b] = 0;
        if (!use[b]) continue;
        if (k[b].lo == EMPTY_KEY && k[b].hi == EMPTY_KEY) {
            if (MIN) atomicMin(t.val_at(t.cap_max), v[b]);
            out[b] = t.cap_max;
            done[b] = true;
        } else {
            slot[b] = (uint32_t)mix64(k[b].lo ^ mix64(k[b].hi)) & mask;
        }
    }
    for (uint32_t probe = 0; probe < cap; ++probe) {
        int seen[B];
#pragma unroll
        for (int b = 0; b < B; ++b)
            seen[b] = done[b] || !PEEK ? PEEK_ASK : peek_slot(t.key_at(slot[b]), k[b]);
        Key128 cur[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            cur[b] = k[b];
            if (!done[b] && seen[b] == PEEK_ASK) cur[b] = atomicCAS(t.key_at(slot[b]), empty, k[b]);
        }
        bool again = false;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            if (done[b]) continue;
            if (seen[b] != PEEK_OTHER && (key_eq(cur[b], empty) || key_eq(cur[b], k[b]))) {
                if (MIN && LOWER) lower_to(t.val_at(slot[b]), v[b]);
                else if (MIN) atomicMin(t.val_at(slot[b]), v[b]);
                out[b] = slot[b];
                if (fresh) fresh[b] = key_eq(cur[b], empty);
                done[b] = true;
            } else {
                slot[b] = (slot[b] + 1) & mask;
                again = true;
            }
        }
        if (!again) break;
    }
}

}  // namespace
}  // namespace prim
}  // namespace odp
