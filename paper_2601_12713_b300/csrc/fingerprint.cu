// fingerprint.cu -- odp_fingerprint: FP128 v1 of a ragged batch of buffers in
// one persistent launch (paper Sec. 5.1 hashes every transferred buffer; this
// is the data-parallel form of that step).
//
// Schedule (none of it changes the result; see the tree argument below):
//   plan     per buffer: chunk count, tile size 2^m_b chunks, tile and node
//            offsets (exclusive scans); tile -> buffer list.
//   tiles    persistent warps take tiles from an atomic counter.  A warp
//            hashes the tile's chunks (lane l loads 16-byte words l + 32j),
//            reduces up to 32 leaves across lanes, folds groups of 32 with
//            a small stack (tiles > 32 chunks), then either finalises the
//            buffer (single-tile buffers) or climbs the upper tree: it
//            stores the tile root, bumps the counter of its 32-node group and
//            the warp that completes a group combines it, level by level.
// An aligned block of 2^k leaves of a left-balanced tree is a complete
// subtree, and the suffix after the last full block is one too, so tiles of
// 2^m chunks and 32-aligned groups of tile roots give the same root as the
// plain recursive split.
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>

#include "common.cuh"
#include "fingerprint.cuh"
#include "fp128.cuh"

namespace odp {
namespace {

using fp::U128;

constexpr uint32_t CHUNK = 4096;
constexpr int MAX_SMALL_PLAN = 8192;  // single-block plan up to this many buffers

struct PlanHeader {
    unsigned long long total_chunks;
    unsigned long long err;  // packed (index, -status) of the first bad buffer
    uint32_t m_floor;
    uint32_t total_tiles;
    uint32_t total_nodes;
    uint32_t tile_counter;
    uint32_t warps_done;   // warps that left the tile loop (reset by the last one)
    uint32_t n_big;        // buffers listed for fp_plan_big
};

struct FpArgs {
    const void* const* ptrs;
    const uint64_t* sizes;
    odp_fp128* out;
    uint32_t n;
    uint32_t tmin;        // target tiles per buffer (launch-level knob)
    uint32_t cap_tiles;   // tile capacity of the scratch
    PlanHeader* hdr;
    uint32_t* tile_off;   // n + 1
    uint32_t* node_off;   // n + 1
    uint32_t* block_sums; // 2 * plan blocks
    uint32_t* tile_buf;   // cap_tiles: the buffer of each tile
    uint32_t* big;        // n: buffers whose later tile entries fp_plan_big writes
    uint32_t* counters;   // 2 * cap_tiles
    U128* nodes;          // 2 * cap_tiles
    int32_t* status;      // per-device status word (null: not published)
    uint32_t single;      // 1: one buffer, planned inside fp_tiles
    uint32_t host_one;    // 1: that buffer is one_ptr / one_size (given by value)
    const void* one_ptr;
    uint64_t one_size;
};

__host__ __device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ uint32_t umin32(uint32_t a, uint32_t b) { return a < b ? a : b; }

__host__ __device__ __forceinline__ uint64_t n_chunks(uint64_t size) {
    return (size + CHUNK - 1) / CHUNK;
}

__host__ __device__ __forceinline__ int ceil_log2(uint64_t v) {
#ifdef __CUDA_ARCH__
    return v <= 1 ? 0 : 64 - __clzll((long long)(v - 1));
#else
    return v <= 1 ? 0 : 64 - __builtin_clzll(v - 1);
#endif
}

// Tile size exponent of a buffer: aim for `tmin` tiles, at most 32 chunks per
// tile unless the scratch capacity forces larger tiles (m_floor).
__host__ __device__ __forceinline__ int tile_log2(uint64_t nchunk, uint32_t tmin, uint32_t m_floor) {
    uint64_t want = (nchunk + tmin - 1) / tmin;
    int m = ceil_log2(want) < 5 ? ceil_log2(want) : 5;
    return m > (int)m_floor ? m : (int)m_floor;
}

__host__ __device__ __forceinline__ uint64_t n_tiles(uint64_t nchunk, int m) {
    return (nchunk + (1ull << m) - 1) >> m;
}

// Nodes kept for the upper tree of a buffer with `nt` tiles (0 if nt <= 1):
// every level down from the tiles, including the single top node.
__device__ __forceinline__ uint64_t n_nodes(uint64_t nt) {
    if (nt <= 1) return 0;
    uint64_t s = 0;
    for (uint64_t l = nt;; l = (l + 31) / 32) {
        s += l;
        if (l == 1) break;
    }
    return s;
}

// --------------------------------------------------------------- plan

// Per-buffer work shared by the plan kernels: chunk count; empty buffers and
// null pointers are finished here.
__device__ __forceinline__ uint64_t plan_chunks(const FpArgs& a, uint32_t i, uint64_t size,
                                                const void* ptr) {
    if (size == 0) {
        U128 e = fp::empty_input();
        a.out[i].lo = e.x;
        a.out[i].hi = e.y;
        return 0;
    }
    if (ptr == nullptr) {
        a.out[i].lo = 0;
        a.out[i].hi = 0;
        record_error(&a.hdr->err, i, ODP_ERR_INVALID_ARG);
        return 0;
    }
    return n_chunks(size);
}

__host__ __device__ __forceinline__ uint32_t floor_for(unsigned long long total_chunks,
                                                       uint32_t budget) {
    uint32_t m = 0;
    while ((total_chunks >> m) > budget) ++m;
    return m;
}

// Single-block plan for small n: reduce, choose m_floor, scan, write offsets.
__global__ void __launch_bounds__(1024) fp_plan_small(FpArgs a) {
    __shared__ uint32_t sm[40];
    __shared__ unsigned long long s_total;
    if (threadIdx.x == 0) s_total = 0;
    __syncthreads();
    unsigned long long local = 0;
    for (uint32_t i = threadIdx.x; i < a.n; i += blockDim.x)
        local += plan_chunks(a, i, a.sizes[i], a.ptrs[i]);
    atomicAdd(&s_total, local);
    __syncthreads();
    const uint32_t budget = a.cap_tiles - a.n;
    const uint32_t m_floor = floor_for(s_total, budget);
    uint32_t base_t = 0, base_n = 0;
    for (uint32_t i0 = 0; i0 < a.n; i0 += blockDim.x) {
        uint32_t i = i0 + threadIdx.x;
        uint32_t nt = 0, nn = 0;
        if (i < a.n) {
            uint64_t size = a.sizes[i];
            if (size != 0 && a.ptrs[i] != nullptr) {
                uint64_t nc = n_chunks(size);
                nt = (uint32_t)n_tiles(nc, tile_log2(nc, a.tmin, m_floor));
                nn = (uint32_t)n_nodes(nt);
            }
        }
        uint32_t tot_t, tot_n;
        uint32_t et = block_exclusive_scan_u32(nt, &tot_t, sm);
        uint32_t en = block_exclusive_scan_u32(nn, &tot_n, sm);
        if (i < a.n) {
            a.tile_off[i] = base_t + et;
            a.node_off[i] = base_n + en;
        }
        base_t += tot_t;
        base_n += tot_n;
    }
    if (threadIdx.x == 0) {
        a.tile_off[a.n] = base_t;
        a.node_off[a.n] = base_n;
        a.hdr->total_chunks = s_total;
        a.hdr->m_floor = m_floor;
        a.hdr->total_tiles = base_t;
        a.hdr->total_nodes = base_n;
        a.hdr->tile_counter = 0;
    }
}

// Multi-block plan, pass 1: total chunk count (and empty-buffer results).
__global__ void __launch_bounds__(256) fp_plan_count(FpArgs a) {
    __shared__ unsigned long long s_total;
    if (threadIdx.x == 0) s_total = 0;
    __syncthreads();
    unsigned long long local = 0;
    const uint32_t base = blockIdx.x * 1024;
    uint64_t sz[4];
    const void* pt[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {  // every load in flight before the first use
        const uint32_t i = base + k * 256 + threadIdx.x;
        sz[k] = i < a.n ? a.sizes[i] : 0;
        pt[k] = i < a.n ? a.ptrs[i] : nullptr;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t i = base + k * 256 + threadIdx.x;
        if (i < a.n) local += plan_chunks(a, i, sz[k], pt[k]);
    }
    atomicAdd(&s_total, local);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(&a.hdr->total_chunks, s_total);
}

// Pass 2: per-buffer tiles/nodes, block-local exclusive offsets, block sums.
__global__ void __launch_bounds__(256) fp_plan_scan(FpArgs a) {
    __shared__ uint32_t sm[40];
    const uint32_t m_floor = floor_for(a.hdr->total_chunks, a.cap_tiles - a.n);
    uint32_t base = blockIdx.x * 1024 + threadIdx.x * 4;
    uint32_t nt[4], nn[4], st = 0, sn = 0;
    for (int k = 0; k < 4; ++k) {
        uint32_t i = base + k;
        nt[k] = nn[k] = 0;
        if (i < a.n) {
            uint64_t size = a.sizes[i];
            if (size != 0 && a.ptrs[i] != nullptr) {
                uint64_t nc = n_chunks(size);
                nt[k] = (uint32_t)n_tiles(nc, tile_log2(nc, a.tmin, m_floor));
                nn[k] = (uint32_t)n_nodes(nt[k]);
            }
        }
        st += nt[k];
        sn += nn[k];
    }
    uint32_t tot_t, tot_n;
    uint32_t et = block_exclusive_scan_u32(st, &tot_t, sm);
    uint32_t en = block_exclusive_scan_u32(sn, &tot_n, sm);
    for (int k = 0; k < 4; ++k) {
        uint32_t i = base + k;
        if (i < a.n) {
            a.tile_off[i] = et;
            a.node_off[i] = en;
        }
        et += nt[k];
        en += nn[k];
    }
    if (threadIdx.x == 0) {
        a.block_sums[2 * blockIdx.x] = tot_t;
        a.block_sums[2 * blockIdx.x + 1] = tot_n;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.hdr->m_floor = m_floor;
}

// Pass 3 (one block): exclusive scan of the block sums; totals.
__global__ void __launch_bounds__(1024) fp_plan_blocks(FpArgs a, uint32_t nblocks) {
    __shared__ uint32_t sm[40];
    uint32_t base_t = 0, base_n = 0;
    for (uint32_t b0 = 0; b0 < nblocks; b0 += blockDim.x) {
        uint32_t b = b0 + threadIdx.x;
        uint32_t vt = b < nblocks ? a.block_sums[2 * b] : 0;
        uint32_t vn = b < nblocks ? a.block_sums[2 * b + 1] : 0;
        uint32_t tt, tn;
        uint32_t et = block_exclusive_scan_u32(vt, &tt, sm);
        uint32_t en = block_exclusive_scan_u32(vn, &tn, sm);
        if (b < nblocks) {
            a.block_sums[2 * b] = base_t + et;
            a.block_sums[2 * b + 1] = base_n + en;
        }
        base_t += tt;
        base_n += tn;
    }
    if (threadIdx.x == 0) {
        a.tile_off[a.n] = base_t;
        a.node_off[a.n] = base_n;
        a.hdr->total_tiles = base_t;
        a.hdr->total_nodes = base_n;
        a.hdr->tile_counter = 0;
    }
}

// A buffer's first REC_DIRECT tile-list entries are written by its thread in
// fp_plan_add; buffers with more tiles are listed, and fp_plan_big writes the
// rest with a warp per buffer.  Most buffers of a ragged batch have one tile.
constexpr uint32_t REC_DIRECT = 4;

// Pass 4: add the block offsets; write the tile list.
__global__ void __launch_bounds__(256) fp_plan_add(FpArgs a) {
    const uint32_t bt = a.block_sums[2 * blockIdx.x], bn = a.block_sums[2 * blockIdx.x + 1];
    const uint32_t m_floor = a.hdr->m_floor;
    const uint32_t base = blockIdx.x * 1024 + threadIdx.x * 4;
    for (int k = 0; k < 4; ++k) {
        const uint32_t i = base + k;
        if (i >= a.n) break;
        const uint32_t t0 = a.tile_off[i] + bt;
        a.tile_off[i] = t0;
        a.node_off[i] += bn;
        const uint64_t size = a.sizes[i];
        if (size == 0 || a.ptrs[i] == nullptr) continue;
        const uint64_t nc = n_chunks(size);
        const uint32_t nt = (uint32_t)n_tiles(nc, tile_log2(nc, a.tmin, m_floor));
        for (uint32_t j = 0; j < nt && j < REC_DIRECT; ++j) a.tile_buf[t0 + j] = i;
        if (nt > REC_DIRECT) a.big[atomicAdd(&a.hdr->n_big, 1u)] = i;
    }
}

// Pass 5 (multi-block plan): the remaining tile-list entries of listed buffers.
__global__ void __launch_bounds__(256) fp_plan_big(FpArgs a) {
    const uint32_t nb = a.hdr->n_big, m_floor = a.hdr->m_floor;
    const int lane = lane_id();
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t q = gw; q < nb; q += nw) {
        const uint32_t i = a.big[q];
        const uint64_t nc = n_chunks(a.sizes[i]);
        const uint32_t nt = (uint32_t)n_tiles(nc, tile_log2(nc, a.tmin, m_floor));
        const uint32_t t0 = a.tile_off[i];
        for (uint32_t j = REC_DIRECT + lane; j < nt; j += 32) a.tile_buf[t0 + j] = i;
    }
}

// Tile list of the one-block plan (binary search over tile offsets).  The
// tree counters need no reset: each group's last arriver sets its counter
// back to zero.
__global__ void __launch_bounds__(256) fp_plan_tiles(FpArgs a) {
    const uint32_t T = a.hdr->total_tiles;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += stride) {
        // largest i with tile_off[i] <= t and a non-empty range
        uint32_t lo = 0, hi = a.n;  // invariant: tile_off[lo] <= t < tile_off[hi]
        while (hi - lo > 1) {
            uint32_t mid = (lo + hi) >> 1;
            if (a.tile_off[mid] <= t) lo = mid; else hi = mid;
        }
        a.tile_buf[t] = lo;
    }
}

// --------------------------------------------------------------- tiles

__device__ __forceinline__ uint4 ld_stream(const uint8_t* p) {
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0, %1, %2, %3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p));
    return v;
}

// Keep the first v (0..16) bytes of a little-endian 16-byte word.
__device__ __forceinline__ uint4 keep_bytes(uint4 w, uint32_t v) {
    uint32_t m[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int k = (int)v - 4 * i;  // valid bytes in component i
        m[i] = k >= 4 ? 0xFFFFFFFFu : (k <= 0 ? 0u : (0xFFFFFFFFu >> (32 - 8 * k)));
    }
    return make_uint4(w.x & m[0], w.y & m[1], w.z & m[2], w.w & m[3]);
}

// 16 bytes starting `off` (1..15) bytes into the 32-byte pair (lo, hi).
__device__ __forceinline__ uint4 funnel16(uint4 lo, uint4 hi, uint32_t off) {
    const uint32_t q = off >> 2, s = (off & 3) * 8;
    uint32_t c0, c1, c2, c3, c4;
    if (q == 0) { c0 = lo.x; c1 = lo.y; c2 = lo.z; c3 = lo.w; c4 = hi.x; }
    else if (q == 1) { c0 = lo.y; c1 = lo.z; c2 = lo.w; c3 = hi.x; c4 = hi.y; }
    else if (q == 2) { c0 = lo.z; c1 = lo.w; c2 = hi.x; c3 = hi.y; c4 = hi.z; }
    else { c0 = lo.w; c1 = hi.x; c2 = hi.y; c3 = hi.z; c4 = hi.w; }
    return make_uint4(__funnelshift_r(c0, c1, s), __funnelshift_r(c1, c2, s),
                      __funnelshift_r(c2, c3, s), __funnelshift_r(c3, c4, s));
}

// Word `wi` of a chunk whose first byte is at `cp`, `r` valid bytes, general
// alignment.  Only aligned 16-byte blocks that hold a valid byte are read.
__device__ __forceinline__ uint4 load_word_general(const uint8_t* cp, uint32_t wi, uint32_t r) {
    const uint32_t o = 16 * wi;
    if (o >= r) return make_uint4(0, 0, 0, 0);
    const uint32_t v = min(16u, r - o);
    const uint8_t* p = cp + o;
    const uint32_t off = (uint32_t)((uintptr_t)p & 15);
    uint4 w;
    if (off == 0) {
        w = ld_stream(p);
    } else {
        const uint8_t* b0 = p - off;
        uint4 lo = ld_stream(b0);
        uint4 hi = make_uint4(0, 0, 0, 0);
        if (off + v > 16) hi = ld_stream(b0 + 16);
        w = funnel16(lo, hi, off);
    }
    return v < 16 ? keep_bytes(w, v) : w;
}

// Chain absorption, lane finish and the 32-lane combine.  Lane 0 ends with
// the chunk root.
__device__ __forceinline__ void absorb_and_combine(const uint4 (&w)[8], uint64_t a, uint64_t b,
                                                   uint64_t& rx, uint64_t& ry) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        uint64_t lo = ((uint64_t)w[j].y << 32) | w[j].x;
        uint64_t hi = ((uint64_t)w[j].w << 32) | w[j].z;
        a = fp::chain(a ^ lo, fp::KA1, fp::KA2);
        b = fp::chain(b ^ hi, fp::KB1, fp::KB2);
    }
    a ^= b * fp::KF1;
    b ^= a * fp::KF2;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t ox = shfl_down64(a, d), oy = shfl_down64(b, d);
        a ^= oy;
        b ^= ox ^ oy;
    }
    rx = a;
    ry = b;
}

// Left-balanced combine of `cnt` (1..32, the same in every lane) nodes held
// by lanes 0..cnt-1, each with its leaf count c.  Every lane returns the root
// and its count.  Levels with d >= cnt combine nothing and are skipped: a
// one-chunk tile (most tiles of a batch of small buffers) then costs no
// node mix at all.
__device__ __forceinline__ U128 warp_tree(U128 v, uint64_t& c, uint32_t cnt, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        if ((uint32_t)d >= cnt) break;
        uint64_t rx = shfl_down64(v.x, d), ry = shfl_down64(v.y, d);
        uint64_t rc = shfl_down64(c, d);
        U128 nd = fp::node(v, U128{rx, ry}, c + rc);
        if ((lane & (2 * d - 1)) == 0 && (uint32_t)(lane + d) < cnt) {
            v = nd;
            c += rc;
        }
    }
    v.x = shfl64(v.x, 0);
    v.y = shfl64(v.y, 0);
    c = shfl64(c, 0);
    return v;
}

struct WarpStack {
    U128 node[40];
    uint64_t count[40];
};

// ---------------------------------------------------- one small buffer
// A buffer of at most ONE_SMALL_CHUNKS chunks whose address and size the
// host knows, hashed by a single block: each warp hashes whole chunks into
// leaves in shared memory, warp g reduces the aligned 32-leaf group g (a
// complete subtree), and warp 0 combines the group roots -- the same
// left-balanced tree as the tiled kernel, with no global counters or fences.
constexpr uint32_t ONE_SMALL_CHUNKS = 64;

__global__ void __launch_bounds__(1024) fp_one_small(const uint8_t* base, uint64_t size,
                                                     odp_fp128* out, int32_t* status) {
    __shared__ U128 leaves[ONE_SMALL_CHUNKS];
    __shared__ U128 groups[ONE_SMALL_CHUNKS / 32];
    __shared__ uint64_t gcount[ONE_SMALL_CHUNKS / 32];
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    if (size == 0 || base == nullptr) {
        if (threadIdx.x == 0) {
            const U128 e = size == 0 ? fp::empty_input() : U128{0, 0};
            out->lo = e.x;
            out->hi = e.y;
            if (size != 0 && status) atomicCAS((int*)status, 0, ODP_ERR_INVALID_ARG);
        }
        return;
    }
    const uint64_t nc = n_chunks(size);
    uint64_t a0, b0;
    fp::lane_init(lane, a0, b0);
    const bool aligned = ((uintptr_t)base & 15) == 0;
    for (uint64_t c = warp; c < nc; c += blockDim.x / 32) {
        const uint8_t* cp = base + c * CHUNK;
        const uint32_t r = (uint32_t)umin64(CHUNK, size - c * CHUNK);
        uint4 w[8];
        if (aligned && r == CHUNK) {
#pragma unroll
            for (int j = 0; j < 8; ++j) w[j] = ld_stream(cp + 16 * (lane + 32 * j));
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) w[j] = load_word_general(cp, lane + 32 * j, r);
        }
        uint64_t rx, ry;
        absorb_and_combine(w, a0, b0, rx, ry);
        rx = shfl64(rx, 0);
        ry = shfl64(ry, 0);
        if (lane == 0) leaves[c] = fp::leaf(rx, ry, r);
    }
    __syncthreads();
    const uint32_t ng = (uint32_t)((nc + 31) / 32);
    if ((uint32_t)warp < ng) {
        const uint32_t gc = (uint32_t)umin64(32, nc - 32ull * warp);
        U128 v = (uint32_t)lane < gc ? leaves[32 * warp + lane] : U128{0, 0};
        uint64_t cc = 1;
        const U128 gr = warp_tree(v, cc, gc, lane);
        if (lane == 0) {
            groups[warp] = gr;
            gcount[warp] = cc;
        }
    }
    __syncthreads();
    if (warp == 0) {
        U128 v = (uint32_t)lane < ng ? groups[lane] : U128{0, 0};
        uint64_t cc = (uint32_t)lane < ng ? gcount[lane] : 0;
        const U128 root = warp_tree(v, cc, ng, lane);
        if (lane == 0) {
            const U128 o = fp::finish(root, size, nc);
            out->lo = o.x;
            out->hi = o.y;
        }
    }
}

// ---------------------------------------------------------------- bulk ring
// Optional load path: whole 4 KiB chunks of 16-byte-aligned buffers are
// copied into a per-warp ring of shared-memory slots with 1D bulk copies
// (cp.async.bulk) that complete on one mbarrier per slot, so a warp keeps
// several chunks in flight without holding them in registers.

struct Ring {
    uint8_t* buf;        // STAGES * 4096 bytes of this warp
    uint64_t* bars;      // STAGES mbarriers
    uint32_t parity;     // expected phase parity per slot (bit s)
    uint32_t pending;    // slots with a copy issued and not yet waited for (bit s)
    bool failed;         // a wait ran out: no further copies, no further hashing
    int32_t* timeout;    // status word set when a wait gives up
};

// A wait for one chunk copy gives up after this long (a 4 KiB copy normally
// lands within microseconds); the warp then stops using its ring.
constexpr uint64_t RING_WAIT_NS = 50ull * 1000 * 1000;

// Bytes each slot's mbarrier expects per chunk copy.  Always CHUNK in the
// library; the bounded-wait test builds the sources with a larger value, so
// that a phase can never complete and every wait runs out with no copy left
// in flight.
#ifndef ODP_RING_TX_BYTES
#define ODP_RING_TX_BYTES CHUNK
#endif

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Every kernel variant starts its ring state here (STAGES = 0 has no slots
// and never fails); the mbarriers are initialised only where slots exist.
__device__ __forceinline__ void ring_init(Ring& r, int stages, int lane) {
    r.parity = 0;
    r.pending = 0;
    r.failed = false;
    if (stages == 0) return;
    if (lane == 0) {
        for (int s = 0; s < stages; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(r.bars + s)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncwarp();
}

// Called by the whole warp: lane 0 starts the copy of one 4 KiB chunk into
// slot s; every lane records the slot as pending.
__device__ __forceinline__ void ring_issue(Ring& r, int s, const uint8_t* src, int lane) {
    if (lane == 0) {
        const uint32_t bar = smem_addr(r.bars + s), dst = smem_addr(r.buf + (size_t)s * CHUNK);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"((uint32_t)ODP_RING_TX_BYTES)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
            ::"r"(dst), "l"(src), "r"(CHUNK), "r"(bar)
            : "memory");
    }
    r.pending |= 1u << s;
}

// Polls slot s's phase until every lane has seen it complete, or until
// RING_WAIT_NS have passed on lane 0's clock (a warp-uniform decision).
__device__ __forceinline__ bool ring_poll(const Ring& r, int s) {
    const uint32_t bar = smem_addr(r.bars + s), par = (r.parity >> s) & 1u;
    uint64_t deadline = 0;
    for (uint32_t it = 1;; ++it) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
            "selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(bar), "r"(par)
            : "memory");
        if (__all_sync(ODP_FULL_MASK, done)) return true;
        if ((it & 63) == 0) {
            const uint64_t now = shfl64(global_ns(), 0);
            if (deadline == 0)
                deadline = now + RING_WAIT_NS;
            else if (now > deadline)
                return false;
        }
    }
}

// All lanes wait for slot s.  A wait that runs out records ODP_ERR_TIMEOUT
// and marks the ring failed; the caller then abandons the tile.
__device__ __forceinline__ bool ring_wait(Ring& r, int s, int lane) {
    if (ring_poll(r, s)) {
        r.parity ^= 1u << s;
        r.pending &= ~(1u << s);
        return true;
    }
    if (lane == 0 && r.timeout) atomicCAS((int*)r.timeout, 0, ODP_ERR_TIMEOUT);
    r.failed = true;
    return false;
}

// Before the warp exits: wait (bounded again) for copies still in flight
// into its ring.  Nothing is pending unless a wait ran out.
__device__ __forceinline__ void ring_drain(Ring& r) {
    for (int s = 0; r.pending != 0 && s < 32; ++s) {
        if (!((r.pending >> s) & 1u)) continue;
        if (ring_poll(r, s)) r.parity ^= 1u << s;
        r.pending &= ~(1u << s);
    }
}

// Hash chunks [c0, c0 + cnt) of a buffer (`cnt` <= 2^m); returns the subtree
// root in every lane.  With STAGES > 0, whole chunks of a 16-byte-aligned
// buffer (all but a partial last one) stream through the warp's bulk ring.
template <bool ALIGNED, int STAGES>
__device__ __forceinline__ U128 hash_tile(const uint8_t* base, uint64_t size, uint64_t c0,
                                          uint64_t cnt, int lane, uint64_t a0, uint64_t b0,
                                          WarpStack* st, Ring& ring) {
    int depth = 0;
    U128 root{0, 0};
    uint64_t root_c = 0;
    uint64_t nbulk = 0;
    if constexpr (STAGES > 0) {
        if (ALIGNED) nbulk = (size - (c0 + cnt - 1) * CHUNK) >= CHUNK ? cnt : cnt - 1;
        for (uint64_t k = 0; k < nbulk && k < (uint64_t)STAGES; ++k)
            ring_issue(ring, (int)k, base + (c0 + k) * CHUNK, lane);
    }
    for (uint64_t g0 = 0; g0 < cnt; g0 += 32) {
        const uint32_t gc = (uint32_t)umin64(32, cnt - g0);
        uint64_t mx = 0, my = 0;
        for (uint32_t k = 0; k < gc; ++k) {
            const uint64_t c = c0 + g0 + k;
            const uint8_t* cp = base + c * CHUNK;
            const uint32_t r = (uint32_t)umin64(CHUNK, size - c * CHUNK);
            uint4 w[8];
            bool from_ring = false;
            if constexpr (STAGES > 0) {
                const uint64_t kk = g0 + k;  // chunk index within the tile
                if (kk < nbulk) {
                    const int slot = (int)(kk % STAGES);
                    if (!ring_wait(ring, slot, lane)) return U128{0, 0};  // timed out
                    const uint8_t* sb = ring.buf + (size_t)slot * CHUNK;
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        w[j] = *reinterpret_cast<const uint4*>(sb + 16 * (lane + 32 * j));
                    __syncwarp();
                    if (kk + STAGES < nbulk)
                        ring_issue(ring, slot, base + (c0 + kk + STAGES) * CHUNK, lane);
                    from_ring = true;
                }
            }
            if (from_ring) {
            } else if (ALIGNED && r == CHUNK) {
#pragma unroll
                for (int j = 0; j < 8; ++j) w[j] = ld_stream(cp + 16 * (lane + 32 * j));
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) w[j] = load_word_general(cp, lane + 32 * j, r);
            }
            uint64_t rx, ry;
            absorb_and_combine(w, a0, b0, rx, ry);
            rx = shfl64(rx, 0);
            ry = shfl64(ry, 0);
            if ((uint32_t)lane == k) {
                mx = rx;
                my = ry;
            }
        }
        // leaves of this group, one per lane, then the group subtree
        const uint64_t cl = c0 + g0 + (uint64_t)umin32(lane, gc - 1);
        const uint64_t rl = umin64(CHUNK, size - cl * CHUNK);
        U128 lf = fp::leaf(mx, my, rl);
        uint64_t lc = 1;
        U128 gr = warp_tree(lf, lc, gc, lane);
        if (cnt <= 32) return gr;
        // push the group root; merge equal-sized neighbours
        if (lane == 0) {
            st->node[depth] = gr;
            st->count[depth] = lc;
        }
        ++depth;
        __syncwarp();
        while (depth >= 2 && st->count[depth - 2] == st->count[depth - 1]) {
            U128 l = st->node[depth - 2], rr = st->node[depth - 1];
            uint64_t cc = st->count[depth - 2] + st->count[depth - 1];
            U128 nd = fp::node(l, rr, cc);
            __syncwarp();
            if (lane == 0) {
                st->node[depth - 2] = nd;
                st->count[depth - 2] = cc;
            }
            --depth;
            __syncwarp();
        }
    }
    // fold right to left
    root = st->node[depth - 1];
    root_c = st->count[depth - 1];
    for (int i = depth - 2; i >= 0; --i) {
        root_c += st->count[i];
        root = fp::node(st->node[i], root, root_c);
    }
    __syncwarp();
    return root;
}

// Where tile t lies: its buffer, the buffer's size and base, and its chunk range.
struct TileInfo {
    const uint8_t* base;
    uint64_t size, nchunk, c0, cnt;
    uint32_t b, tb;
    int m;
};

__device__ __forceinline__ TileInfo finish_info(TileInfo ti, const FpArgs& a, uint32_t m_floor) {
    ti.nchunk = n_chunks(ti.size);
    ti.m = tile_log2(ti.nchunk, a.tmin, m_floor);
    ti.c0 = (uint64_t)ti.tb << ti.m;
    ti.cnt = umin64(1ull << ti.m, ti.nchunk - ti.c0);
    return ti;
}

// Tile t of a planned batch: its buffer from the tile list.
__device__ __forceinline__ TileInfo batch_info(const FpArgs& a, uint32_t t, uint32_t m_floor) {
    TileInfo ti;
    ti.b = a.tile_buf[t];
    ti.tb = t - a.tile_off[ti.b];
    ti.size = a.sizes[ti.b];
    ti.base = (const uint8_t*)a.ptrs[ti.b];
    return finish_info(ti, a, m_floor);
}

// Tile t of the one buffer of a single-buffer call (no plan, no tile list).
__device__ __forceinline__ TileInfo single_info(const FpArgs& a, uint32_t t, uint32_t m_floor) {
    TileInfo ti;
    ti.b = 0;
    ti.tb = t;
    ti.size = a.host_one ? a.one_size : a.sizes[0];
    ti.base = (const uint8_t*)(a.host_one ? a.one_ptr : a.ptrs[0]);
    return finish_info(ti, a, m_floor);
}

// Finishes a buffer of one tile, or climbs the 32-ary groups of tile roots:
// the last warp to arrive at a group combines it (level L holds nodes
// covering 2^m * 32^L chunks) and the last one at the top finishes the hash.
__device__ __forceinline__ void climb(const FpArgs& a, const TileInfo& ti, U128 root, int lane) {
    const uint64_t ntile = n_tiles(ti.nchunk, ti.m);
    if (ntile == 1) {
        if (lane == 0) {
            U128 o = fp::finish(root, ti.size, ti.nchunk);
            a.out[ti.b].lo = o.x;
            a.out[ti.b].hi = o.y;
        }
        return;
    }
    uint64_t nl = ntile, idx = ti.tb, off = a.single ? 0 : a.node_off[ti.b];
    uint64_t span = 1ull << ti.m;
    U128 node = root;
    while (true) {
        if (nl == 1) {
            if (lane == 0) {
                U128 o = fp::finish(node, ti.size, ti.nchunk);
                a.out[ti.b].lo = o.x;
                a.out[ti.b].hi = o.y;
            }
            return;
        }
        const uint64_t nup = (nl + 31) / 32;
        const uint64_t g = idx / 32;
        const uint32_t gsize = (uint32_t)umin64(32, nl - 32 * g);
        uint32_t old = 0;
        if (lane == 0) {
            a.nodes[off + idx] = node;
            __threadfence();
            old = atomicAdd(&a.counters[off + nl + g], 1u);
        }
        old = __shfl_sync(ODP_FULL_MASK, old, 0);
        if (old != gsize - 1) return;  // another warp finishes this group
        __threadfence();
        U128 v{0, 0};
        uint64_t c = 0;
        if ((uint32_t)lane < gsize) {
            const U128* src = &a.nodes[off + 32 * g + lane];
            v.x = __ldcg((const unsigned long long*)&src->x);
            v.y = __ldcg((const unsigned long long*)&src->y);
            const uint64_t first = (32 * g + lane) * span;
            c = umin64(span, ti.nchunk - first);
        }
        if (lane == 0) a.counters[off + nl + g] = 0;  // ready for the next call
        node = warp_tree(v, c, gsize, lane);
        off += nl;
        nl = nup;
        idx = g;
        span *= 32;
    }
}

// Resident warps per SM the register budget is set for: the register-load
// path (STAGES = 0) needs more warps in flight than the bulk-copy ring.
template <int WARPS, int STAGES>
constexpr int fp_min_ctas() {
    return (STAGES == 0 ? 24 : 16) / WARPS > 0 ? (STAGES == 0 ? 24 : 16) / WARPS : 1;
}

template <int WARPS, int STAGES>
__global__ void __launch_bounds__(WARPS * 32, fp_min_ctas<WARPS, STAGES>()) fp_tiles(FpArgs a) {
    __shared__ WarpStack stacks[WARPS];
    extern __shared__ __align__(128) uint8_t ring_smem[];
    const int lane = lane_id();
    const int warp = threadIdx.x >> 5;
    WarpStack* st = &stacks[warp];
    Ring ring;
    ring.buf = ring_smem + (size_t)warp * STAGES * CHUNK;
    ring.bars = reinterpret_cast<uint64_t*>(ring_smem + (size_t)WARPS * STAGES * CHUNK) + warp * 8;
    ring.timeout = a.status;
    ring_init(ring, STAGES, lane);
    uint64_t a0, b0;
    fp::lane_init(lane, a0, b0);
    uint32_t T, m_floor;
    if (a.single) {
        // one buffer: the plan is a few integer operations, done by every warp
        const uint64_t size = a.host_one ? a.one_size : a.sizes[0];
        const bool null_ptr = (a.host_one ? a.one_ptr : a.ptrs[0]) == nullptr;
        if (size == 0 || null_ptr) {
            T = 0;
            m_floor = 0;
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                U128 e = size == 0 ? fp::empty_input() : U128{0, 0};
                a.out[0].lo = e.x;
                a.out[0].hi = e.y;
                if (size != 0 && a.status) atomicCAS((int*)a.status, 0, ODP_ERR_INVALID_ARG);
            }
        } else {
            const uint64_t nc = n_chunks(size);
            m_floor = floor_for(nc, a.cap_tiles - 1);
            T = (uint32_t)n_tiles(nc, tile_log2(nc, a.tmin, m_floor));
        }
    } else {
        T = a.hdr->total_tiles;
        m_floor = a.hdr->m_floor;
    }

    // A warp's first tile is its global warp index and its second that plus
    // the warp count; later tiles come from the shared counter, requested
    // when the previous tile starts so the atomic (contended by every warp)
    // completes while a tile is hashed.  Warps without a first tile exit at
    // once and never touch the counter, so a small buffer costs a few
    // atomics, not one per warp of the grid.
    const uint32_t total = gridDim.x * WARPS;
    uint32_t t = blockIdx.x * WARPS + warp;
    if (t >= T) {
        // no tiles at all (empty or null buffers only): publish the plan's error here
        if (T == 0 && t == 0 && lane == 0 && !a.single && a.status) {
            const unsigned long long e = a.hdr->err;
            if (e != ~0ull) atomicCAS((int*)a.status, 0, -(int)(e & 0xFF));
        }
        return;
    }
    uint32_t t_next = t + total;
    bool first = true;
    while (t < T) {
        if (!first && lane == 0) t_next = 2 * total + atomicAdd(&a.hdr->tile_counter, 1u);
        first = false;
        const TileInfo cur = a.single ? single_info(a, t, m_floor) : batch_info(a, t, m_floor);
        U128 root{0, 0};
        // After a bulk-copy wait ran out (ODP_ERR_TIMEOUT is recorded) the
        // warp hashes nothing more, but still climbs, so every tree counter
        // and the tile counter end the call reset for the next one.
        if (ring.failed) {
        } else if (((uintptr_t)cur.base & 15) == 0) {
            root = hash_tile<true, STAGES>(cur.base, cur.size, cur.c0, cur.cnt, lane, a0, b0, st, ring);
        } else {
            root = hash_tile<false, STAGES>(cur.base, cur.size, cur.c0, cur.cnt, lane, a0, b0, st, ring);
        }
        climb(a, cur, root, lane);
        t = __shfl_sync(ODP_FULL_MASK, t_next, 0);
    }
    if constexpr (STAGES > 0) ring_drain(ring);
    // The last warp out (of the min(T, warps) that took tiles) resets the
    // tile counter for the next call and publishes the plan's error code (the
    // first error index is not kept).
    if (lane == 0) {
        __threadfence();
        const uint32_t takers = T < total ? T : total;
        if (atomicAdd(&a.hdr->warps_done, 1u) == takers - 1) {
            a.hdr->tile_counter = 0;
            a.hdr->warps_done = 0;
            if (!a.single && a.status) {
                const unsigned long long e = a.hdr->err;
                if (e != ~0ull) atomicCAS((int*)a.status, 0, -(int)(e & 0xFF));
            }
        }
    }
}

}  // namespace

template <int W, int S>
static size_t fp_dyn_smem() {
    return S > 0 ? (size_t)W * S * CHUNK + (size_t)W * 64 : 0;
}

template <int W, int S>
static int fp_prepare() {
    // opt in to more than 48 KiB of dynamic shared memory, once per device
    static std::atomic<bool> done[256] = {};
    const int dev = current_device();
    if (S > 0 && dev < 256 && !done[dev].load(std::memory_order_acquire)) {
        if (cudaFuncSetAttribute(fp_tiles<W, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fp_dyn_smem<W, S>()) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        done[dev].store(true, std::memory_order_release);
    }
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fp_tiles<W, S>, W * 32, fp_dyn_smem<W, S>());
    return std::max(1, occ);
}

template <int W, int S>
static void fp_tiles_launch(const FpArgs& a, int grid, cudaStream_t stream) {
    fp_tiles<W, S><<<grid, W * 32, fp_dyn_smem<W, S>(), stream>>>(a);
}

// The (warps per CTA, stages) pairs that are instantiated.
static bool fp_variant_ok(int W, int S) {
    return (W == 4 || W == 8 || W == 16) && (S == 0 || S == 2 || S == 4) && !(W == 16 && S == 4);
}

static int fp_occupancy(int W, int S) {
    switch (W * 16 + S) {
        case 4 * 16 + 0: return fp_prepare<4, 0>();
        case 4 * 16 + 2: return fp_prepare<4, 2>();
        case 4 * 16 + 4: return fp_prepare<4, 4>();
        case 8 * 16 + 2: return fp_prepare<8, 2>();
        case 8 * 16 + 4: return fp_prepare<8, 4>();
        case 16 * 16 + 0: return fp_prepare<16, 0>();
        case 16 * 16 + 2: return fp_prepare<16, 2>();
        default: return fp_prepare<8, 0>();
    }
}

static void fp_launch(const FpArgs& a, int W, int S, int grid, cudaStream_t stream) {
    switch (W * 16 + S) {
        case 4 * 16 + 0: fp_tiles_launch<4, 0>(a, grid, stream); break;
        case 4 * 16 + 2: fp_tiles_launch<4, 2>(a, grid, stream); break;
        case 4 * 16 + 4: fp_tiles_launch<4, 4>(a, grid, stream); break;
        case 8 * 16 + 2: fp_tiles_launch<8, 2>(a, grid, stream); break;
        case 8 * 16 + 4: fp_tiles_launch<8, 4>(a, grid, stream); break;
        case 16 * 16 + 0: fp_tiles_launch<16, 0>(a, grid, stream); break;
        case 16 * 16 + 2: fp_tiles_launch<16, 2>(a, grid, stream); break;
        default: fp_tiles_launch<8, 0>(a, grid, stream); break;
    }
}

// Bytes at the start of each plan scratch block known to be zero (header +
// tree counters), per block address.
static std::mutex g_zero_mu;
static std::map<void*, size_t> g_zeroed;

// Byte offsets of the plan's arrays in its scratch block, for nn buffers.
struct PlanLayout {
    size_t hdr, cnt, zero_needed, toff, noff, bsum, big, tbuf, nodes, bytes;
};

static PlanLayout plan_layout(uint32_t nn) {
    const uint32_t cap_tiles = nn + (1u << 20);
    const uint32_t nblocks = (nn + 1023) / 1024;
    PlanLayout p{};
    size_t bytes = 0;
    auto carve = [&](size_t sz) {
        size_t o = bytes;
        bytes = align_up(bytes + sz, 256);
        return o;
    };
    // The header and the tree counters sit at fixed places in front, so a
    // call with another n finds its counters inside the region earlier calls
    // left at zero (the last arriver of every group resets its counter).
    p.hdr = carve(sizeof(PlanHeader));
    p.cnt = carve(sizeof(uint32_t) * 2 * (size_t)cap_tiles);
    p.zero_needed = bytes;
    p.toff = carve(sizeof(uint32_t) * (nn + 1));
    p.noff = carve(sizeof(uint32_t) * (nn + 1));
    p.bsum = carve(sizeof(uint32_t) * 2 * (nblocks + 1));
    p.big = carve(sizeof(uint32_t) * (nn + 1));
    p.tbuf = carve(sizeof(uint32_t) * (size_t)cap_tiles);
    p.nodes = carve(sizeof(U128) * 2 * (size_t)cap_tiles);
    p.bytes = bytes;
    return p;
}

size_t fp_plan_scratch_bytes(uint64_t n) {
    if (n > (1ull << 28)) n = 1ull << 28;  // larger calls are refused
    return scratch_block_bytes(plan_layout((uint32_t)n).bytes);
}

int fp_run(const void* const* ptrs, const uint64_t* sizes, uint64_t n, odp_fp128* out,
           cudaStream_t stream, const FpLaunch& L, const void* one_ptr, uint64_t one_size) {
    const bool host_one = ptrs == nullptr && sizes == nullptr && n == 1;
    if (n == 0) return ODP_OK;
    if ((!host_one && (!ptrs || !sizes)) || !out) return ODP_ERR_INVALID_ARG;
    if (host_one && n_chunks(one_size) <= ONE_SMALL_CHUNKS) {
        int st = ODP_OK;
        int32_t* status = device_status_word(&st);
        if (!status) return st;
        fp_one_small<<<1, 1024, 0, stream>>>((const uint8_t*)one_ptr, one_size, out, status);
        return cuda_status(cudaGetLastError());
    }
    if (n > (1ull << 28)) return ODP_ERR_UNSUPPORTED;
    int st = ODP_OK;
    int32_t* status = device_status_word(&st);
    if (!status) return st;

    const uint32_t nn = (uint32_t)n;
    const uint32_t cap_tiles = nn + (1u << 20);
    const uint32_t nblocks = (nn + 1023) / 1024;
    const PlanLayout lay = plan_layout(nn);
    const size_t bytes = lay.bytes, zero_needed = lay.zero_needed;
    const size_t o_hdr = lay.hdr, o_cnt = lay.cnt, o_toff = lay.toff, o_noff = lay.noff;
    const size_t o_bsum = lay.bsum, o_tbuf = lay.tbuf, o_nodes = lay.nodes;
    bool fresh = false;
    uint8_t* s = (uint8_t*)scratch_get(SLOT_FP_PLAN, bytes, stream, &st, &fresh);
    if (!s) return st;
    {
        // extend the zeroed prefix (header + counters) when this call needs more
        std::lock_guard<std::mutex> lk(g_zero_mu);
        size_t& z = g_zeroed[s];
        if (fresh) z = 0;
        if (z < zero_needed) {
            ODP_CHECK_CUDA(cudaMemsetAsync(s + z, 0, zero_needed - z, stream));
            z = zero_needed;
        }
    }

    const int sms = device_sm_count();
    FpArgs a;
    a.ptrs = ptrs;
    a.sizes = sizes;
    a.out = out;
    a.n = nn;
    a.cap_tiles = cap_tiles;
    a.hdr = (PlanHeader*)(s + o_hdr);
    a.tile_off = (uint32_t*)(s + o_toff);
    a.node_off = (uint32_t*)(s + o_noff);
    a.block_sums = (uint32_t*)(s + o_bsum);
    a.tile_buf = (uint32_t*)(s + o_tbuf);
    a.big = (uint32_t*)(s + lay.big);
    a.counters = (uint32_t*)(s + o_cnt);
    a.nodes = (U128*)(s + o_nodes);
    a.status = status;
    a.single = nn == 1;
    a.host_one = host_one;
    a.one_ptr = one_ptr;
    a.one_size = one_size;

    const bool ok = fp_variant_ok(L.warps_per_cta, L.stages);
    const int W = ok ? L.warps_per_cta : TILE_WARPS;
    const int S = ok ? L.stages : 0;
    const int occ = fp_occupancy(W, S);
    const int ctas = L.ctas_per_sm > 0 ? std::min(L.ctas_per_sm, occ) : occ;
    const uint64_t total_warps = (uint64_t)sms * ctas * W;
    a.tmin = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(1u << 30,
                                          (uint64_t)L.tmin_scale * total_warps / nn));

    if (!a.single) {
        ODP_CHECK_CUDA(cudaMemsetAsync(a.hdr, 0, sizeof(PlanHeader), stream));
        ODP_CHECK_CUDA(cudaMemsetAsync(&a.hdr->err, 0xFF, sizeof(unsigned long long), stream));
        if (nn <= (uint32_t)MAX_SMALL_PLAN) {
            fp_plan_small<<<1, 1024, 0, stream>>>(a);
        } else {
            fp_plan_count<<<nblocks, 256, 0, stream>>>(a);
            fp_plan_scan<<<nblocks, 256, 0, stream>>>(a);
            fp_plan_blocks<<<1, 1024, 0, stream>>>(a, nblocks);
            fp_plan_add<<<nblocks, 256, 0, stream>>>(a);
            fp_plan_big<<<sms * 4, 256, 0, stream>>>(a);
        }
        if (nn <= (uint32_t)MAX_SMALL_PLAN) fp_plan_tiles<<<sms * 4, 256, 0, stream>>>(a);
    }
    int grid = sms * ctas;
    if (host_one) {
        // the buffer is known here: launch only the warps that get a tile
        const uint64_t nc = n_chunks(one_size);
        const uint64_t T = nc ? n_tiles(nc, tile_log2(nc, a.tmin, floor_for(nc, cap_tiles - 1))) : 0;
        grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(grid, (T + W - 1) / W));
    }
    fp_launch(a, W, S, grid, stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        {
            std::lock_guard<std::mutex> lk(g_zero_mu);
            g_zeroed.erase(s);
        }
        release_slot(SLOT_FP_PLAN, stream);  // counters may be left set
        return ODP_ERR_CUDA;
    }
    return ODP_OK;
}

}  // namespace odp

extern "C" int odp_fingerprint(const void* const* ptrs, const uint64_t* sizes, uint64_t n,
                               odp_fp128* out128, cudaStream_t stream) {
    if (!ptrs || !sizes) return n == 0 ? ODP_OK : ODP_ERR_INVALID_ARG;
    odp::FpLaunch L = odp::fp_schedule_for(n);
    return odp::fp_run(ptrs, sizes, n, out128, stream, L);
}

extern "C" int odp_fingerprint_one(const void* ptr, uint64_t size, odp_fp128* out128,
                                   cudaStream_t stream) {
    if (!out128) return ODP_ERR_INVALID_ARG;
    odp::FpLaunch L = odp::fp_schedule_for(1);
    return odp::fp_run(nullptr, nullptr, 1, out128, stream, L, ptr, size);
}

// ---------------------------------------------------------------------------
// odp_fingerprint_log: the fingerprint of every transfer of an event log,
// written into the transfer's record, in one batched odp_fingerprint call.
// ---------------------------------------------------------------------------
namespace odp {
namespace {

__device__ __forceinline__ bool log_is_transfer(const uint8_t* ev, uint64_t i) {
    const uint32_t k = ev[64 * i + 60];
    return k == ODP_TO_DEV || k == ODP_FROM_DEV || k == ODP_DEV_TO_DEV;
}

// Buffer list of the batched call: a transfer's payload and byte count, an
// empty buffer for every other record.
__global__ void __launch_bounds__(256) fp_log_prep(const uint8_t* ev, const void* const* payloads,
                                                   uint64_t n, const void** ptrs,
                                                   uint64_t* sizes) {
    for (uint64_t i = blockIdx.x * 256ull + threadIdx.x; i < n; i += gridDim.x * 256ull) {
        const bool x = log_is_transfer(ev, i);
        ptrs[i] = x ? payloads[i] : nullptr;
        sizes[i] = x ? reinterpret_cast<const uint64_t*>(ev + 64 * i)[4] : 0;
    }
}

// Fingerprints into the records' fp_lo / fp_hi words (transfers only).
__global__ void __launch_bounds__(256) fp_log_store(uint8_t* ev, const odp_fp128* fps,
                                                    uint64_t n) {
    for (uint64_t i = blockIdx.x * 256ull + threadIdx.x; i < n; i += gridDim.x * 256ull) {
        if (!log_is_transfer(ev, i)) continue;
        uint64_t* r = reinterpret_cast<uint64_t*>(ev + 64 * i);
        const odp_fp128 f = fps[i];
        r[5] = f.lo;
        r[6] = f.hi;
    }
}

}  // namespace

static int fp_run_log(odp_event* events, const void* const* payloads, uint64_t n,
                      cudaStream_t stream) {
    if (n == 0) return ODP_OK;
    if (!events || !payloads) return ODP_ERR_INVALID_ARG;
    if (((uintptr_t)events & 7) != 0) return ODP_ERR_INVALID_ARG;
    if (n > (1ull << 28)) return ODP_ERR_UNSUPPORTED;
    int st = ODP_OK;
    const size_t o_sizes = align_up(8 * n, 256), o_fps = o_sizes + align_up(8 * n, 256);
    uint8_t* s = (uint8_t*)scratch_get(SLOT_FP_LOG, o_fps + 16 * n, stream, &st);
    if (!s) return st;
    const void** ptrs = (const void**)s;
    uint64_t* sizes = (uint64_t*)(s + o_sizes);
    odp_fp128* fps = (odp_fp128*)(s + o_fps);
    const int grid = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)device_sm_count() * 8);
    fp_log_prep<<<grid, 256, 0, stream>>>((const uint8_t*)events, payloads, n, ptrs, sizes);
    ODP_CHECK_CUDA(cudaGetLastError());
    st = fp_run(ptrs, sizes, n, fps, stream, fp_schedule_for(n));
    if (st != ODP_OK) return st;
    fp_log_store<<<grid, 256, 0, stream>>>((uint8_t*)events, fps, n);
    return cuda_status(cudaGetLastError());
}

}  // namespace odp

extern "C" int odp_fingerprint_log(odp_event* events, const void* const* payloads, uint64_t n,
                                   cudaStream_t stream) {
    return odp::fp_run_log(events, payloads, n, stream);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of odp_fingerprint (no counterpart in the paper).
//
// For callers that cannot allocate device memory -- for example code running
// inside a custom allocator or an out-of-memory handler, or an embedding
// that forbids cudaMalloc after start-up.  The plan, tile list, tree nodes
// and counters live in one file-scope device array of fixed size, which every
// GPU that loads the library holds until the process exits.
// ---------------------------------------------------------------------------
#include <map>
#include <mutex>

namespace odp {
namespace {

constexpr uint32_t NA_MAX_BUFFERS = 4096;
constexpr uint32_t NA_CAP_TILES = NA_MAX_BUFFERS + 16384;

constexpr size_t na_up(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t NA_O_HDR = 0;
constexpr size_t NA_O_TOFF = na_up(NA_O_HDR + sizeof(PlanHeader));
constexpr size_t NA_O_NOFF = na_up(NA_O_TOFF + 4ull * (NA_MAX_BUFFERS + 1));
constexpr size_t NA_O_BSUM = na_up(NA_O_NOFF + 4ull * (NA_MAX_BUFFERS + 1));
constexpr size_t NA_O_TBUF = na_up(NA_O_BSUM + 4ull * 2 * 8);
constexpr size_t NA_O_CNT = na_up(NA_O_TBUF + 4ull * NA_CAP_TILES);
constexpr size_t NA_O_NODES = na_up(NA_O_CNT + 4ull * 2 * NA_CAP_TILES);
constexpr size_t NA_BYTES = na_up(NA_O_NODES + sizeof(U128) * 2 * NA_CAP_TILES);

__device__ __align__(256) uint8_t g_na_scratch[NA_BYTES];

std::mutex g_na_mu;
std::map<int, uint8_t*> g_na_base;  // device -> address of g_na_scratch

// Device address of the array on the current device (looked up once per
// device with that device current).  The address is kept for the life of
// the process, so it is stale after cudaDeviceReset (which destroys the
// context holding the array).
uint8_t* na_base(int* status) {
    int dev = current_device();
    std::lock_guard<std::mutex> lk(g_na_mu);
    auto it = g_na_base.find(dev);
    if (it != g_na_base.end()) return it->second;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        *status = ODP_ERR_CUDA;
        return nullptr;
    }
    g_na_base[dev] = (uint8_t*)p;
    return (uint8_t*)p;
}

}  // namespace

static int fp_run_noalloc(const void* const* ptrs, const uint64_t* sizes, uint64_t n,
                          odp_fp128* out, cudaStream_t stream) {
    if (n == 0) return ODP_OK;
    if (!ptrs || !sizes || !out) return ODP_ERR_INVALID_ARG;
    if (n > NA_MAX_BUFFERS) return ODP_ERR_UNSUPPORTED;
    int st = ODP_OK;
    uint8_t* s = na_base(&st);
    if (!s) return st;

    FpArgs a;
    a.ptrs = ptrs;
    a.sizes = sizes;
    a.out = out;
    a.n = (uint32_t)n;
    a.cap_tiles = NA_CAP_TILES;
    a.hdr = (PlanHeader*)(s + NA_O_HDR);
    a.tile_off = (uint32_t*)(s + NA_O_TOFF);
    a.node_off = (uint32_t*)(s + NA_O_NOFF);
    a.block_sums = (uint32_t*)(s + NA_O_BSUM);
    a.tile_buf = (uint32_t*)(s + NA_O_TBUF);
    a.big = nullptr;  // the one-block plan writes the whole tile list in fp_plan_tiles
    a.counters = (uint32_t*)(s + NA_O_CNT);
    a.nodes = (U128*)(s + NA_O_NODES);
    a.status = nullptr;
    a.single = 0;
    a.host_one = 0;
    a.one_ptr = nullptr;
    a.one_size = 0;

    const int sms = device_sm_count();
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fp_tiles<TILE_WARPS, 0>, TILE_WARPS * 32, 0);
    const int ctas = std::max(1, occ);
    const uint32_t total_warps = (uint32_t)(sms * ctas * TILE_WARPS);
    a.tmin = std::max<uint32_t>(1, (uint32_t)(2ull * total_warps / a.n));

    // The header (chunk total, error word, tile counter) and the tree
    // counters (160 KiB) start cleared on every call: a call that overlapped
    // another one, or a launch that failed, may have left a counter set, and
    // that must not spoil the calls after it.  The plan kernels rewrite every
    // offset and the tile list.
    ODP_CHECK_CUDA(cudaMemsetAsync(a.hdr, 0, sizeof(PlanHeader), stream));
    ODP_CHECK_CUDA(cudaMemsetAsync(&a.hdr->err, 0xFF, sizeof(unsigned long long), stream));
    ODP_CHECK_CUDA(cudaMemsetAsync(a.counters, 0, 4ull * 2 * NA_CAP_TILES, stream));
    fp_plan_small<<<1, 1024, 0, stream>>>(a);
    fp_plan_tiles<<<sms * 4, 256, 0, stream>>>(a);
    fp_tiles<TILE_WARPS, 0><<<sms * ctas, TILE_WARPS * 32, 0, stream>>>(a);
    return cuda_status(cudaGetLastError());
}

}  // namespace odp

extern "C" int odp_fingerprint_noalloc(const void* const* ptrs, const uint64_t* sizes,
                                       uint64_t n, odp_fp128* out128, cudaStream_t stream) {
    return odp::fp_run_noalloc(ptrs, sizes, n, out128, stream);
}
